"""Python binding of librca with the C names (include/rca.h).

Argument marshalling only: buffers are torch tensors (or raw integer device
pointers), passed by address; every computation runs in librca's kernels.
Non-zero statuses raise :class:`RcaError` carrying rca_last_error().
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import (LOC2D, LOC3D, rca_batch_item, rca_bf_params, rca_geometry_desc, ulm_cnn_desc,  # noqa: F401
                   ulm_params)


class RcaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)} ({status}): {message}")
        self.status = status


def _status_name(s: int) -> str:
    return L.load().rca_status_string(s).decode()


def _check(st: int, h=None, what: str = ""):
    if st != L.RCA_OK:
        msg = L.load().rca_last_error(h).decode() if h is not None else what
        raise RcaError(st, msg or what)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, C.c_void_p):
        return x
    return C.c_void_p(int(x))


def rca_version() -> int:
    return L.load().rca_version()


def rca_status_string(s: int) -> str:
    return _status_name(s)


def rca_create(device: int = 0):
    h = C.c_void_p()
    _check(L.load().rca_create(C.byref(h), device), None, f"rca_create(device={device})")
    return h


def rca_destroy(h):
    _check(L.load().rca_destroy(h), None, "rca_destroy")


def rca_set_stream(h, stream=None):
    """stream: torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default)."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(L.load().rca_set_stream(h, C.c_void_p(raw) if raw else None), h)


def rca_last_error(h) -> str:
    return L.load().rca_last_error(h).decode()


def rca_sync_status(h) -> int:
    dev = C.c_int(0)
    _check(L.load().rca_sync_status(h, C.byref(dev)), h)
    return dev.value


def rca_reserve(h, g, n_frames: int):
    _check(L.load().rca_reserve(h, g, n_frames), h)


def geometry_desc(geom):
    """rca_geometry_desc from any object with the geometry attributes
    (n_el, nz, ns, P, K, us, pitch, fc, fs, c, z0, dz, fnum, ang_rc, ang_cr).
    Returns (desc, keep-alive arrays)."""
    rc = np.ascontiguousarray(geom.ang_rc, dtype=np.float64)
    cr = np.ascontiguousarray(geom.ang_cr, dtype=np.float64)
    d = rca_geometry_desc()
    d.n_el, d.nz, d.ns, d.P, d.K, d.us = geom.n_el, geom.nz, geom.ns, geom.P, len(rc), geom.us
    d.pitch_m, d.fc_hz, d.fs_hz, d.c_mps = geom.pitch, geom.fc, geom.fs, geom.c
    d.z0_m, d.dz_m, d.fnum = geom.z0, geom.dz, geom.fnum
    d.ang_rc_rad = rc.ctypes.data_as(C.POINTER(C.c_double))
    d.ang_cr_rad = cr.ctypes.data_as(C.POINTER(C.c_double))
    return d, (rc, cr)


def rca_geometry_create(h, geom):
    d, keep = geometry_desc(geom)
    g = C.c_void_p()
    _check(L.load().rca_geometry_create(h, C.byref(d), C.byref(g)), h)
    del keep
    return g


def rca_geometry_destroy(g):
    L.load().rca_geometry_destroy(g)


def rca_delay_tables(h, g):
    t = C.c_void_p()
    _check(L.load().rca_delay_tables(h, g, C.byref(t)), h)
    return t


def rca_tables_destroy(t):
    L.load().rca_tables_destroy(t)


_TABLE_DTYPE = {
    L.RCA_TAB_TX_F64: np.float64, L.RCA_TAB_RX_F64: np.float64, L.RCA_TAB_TX_Q16: np.int32,
    L.RCA_TAB_RX_Q16: np.int32, L.RCA_TAB_W: np.complex64, L.RCA_TAB_DMAX: np.int32,
    L.RCA_TAB_S2_SHIFT: np.float64, L.RCA_TAB_S2_PSI: np.complex64, L.RCA_TAB_S2_EC: np.complex64,
    L.RCA_TAB_S2_COEF: np.complex64, L.RCA_TAB_S2_TMIN: np.int32,
}


def rca_tables_query(t, table_id: int):
    nbytes = C.c_size_t(0)
    dims = (C.c_int * 4)()
    _check(L.load().rca_tables_query(t, table_id, C.byref(nbytes), dims), None, "rca_tables_query")
    return nbytes.value, tuple(d for d in dims if d)


def rca_tables_download(t, table_id: int) -> np.ndarray:
    nbytes, dims = rca_tables_query(t, table_id)
    out = np.zeros(dims, dtype=_TABLE_DTYPE[table_id])
    assert out.nbytes == nbytes, (out.nbytes, nbytes)
    _check(L.load().rca_tables_download(t, table_id, out.ctypes.data_as(C.c_void_p), nbytes), None,
           "rca_tables_download")
    return out


def rca_ingest(h, t, rf, rf_dtype, scale, n_frames, clutter, iq, iq_dtype):
    _check(L.load().rca_ingest(h, t, _ptr(rf), rf_dtype, _ptr(scale), n_frames, clutter, _ptr(iq), iq_dtype), h)


def rca_stage1(h, t, iq, iq_dtype, n_frames, slices):
    _check(L.load().rca_stage1(h, t, _ptr(iq), iq_dtype, n_frames, _ptr(slices)), h)


def rca_stage2_project(h, t, slices, n_frames, planes, planes_dtype):
    _check(L.load().rca_stage2_project(h, t, _ptr(slices), n_frames, _ptr(planes), planes_dtype), h)


def rca_direct_project(h, t, iq, iq_dtype, n_frames, planes, planes_dtype):
    _check(L.load().rca_direct_project(h, t, _ptr(iq), iq_dtype, n_frames, _ptr(planes), planes_dtype), h)


def bf_params(mode=L.RCA_MODE_TWO_STAGE, clutter=L.RCA_CLUTTER_MEAN, iq_dtype=L.RCA_C32, svd_rank=0,
              svd_iterations=0) -> rca_bf_params:
    p = rca_bf_params()
    p.mode, p.clutter, p.iq_dtype = mode, clutter, iq_dtype
    p.svd_rank, p.svd_iterations = svd_rank, svd_iterations
    return p


def rca_beamform_projections(h, t, rf, rf_dtype, scale, n_frames, prm: rca_bf_params, planes, planes_dtype):
    _check(L.load().rca_beamform_projections(h, t, _ptr(rf), rf_dtype, _ptr(scale), n_frames, C.byref(prm),
                                             _ptr(planes), planes_dtype), h)


def make_ulm_params(d=5, sig_z=1.0, sig_lat=1.0, alpha=0.1, ncc_min=0.5, enh=L.ULM_ENH_XDOPPLER) -> ulm_params:
    p = ulm_params()
    p.d, p.sig_z, p.sig_lat, p.alpha, p.ncc_min, p.enh = d, sig_z, sig_lat, alpha, ncc_min, enh
    return p


def ulm_enhance(h, t, planes, planes_dtype, n_frames, enh, A, M):
    _check(L.load().ulm_enhance(h, t, _ptr(planes), planes_dtype, n_frames, enh, _ptr(A), _ptr(M)), h)


def ulm_detect2d(h, t, A, M, n_frames, prm: ulm_params, out2d, cap2d, n2d, ncc_out=None, plane_offsets=None):
    _check(L.load().ulm_detect2d(h, t, _ptr(A), _ptr(M), n_frames, C.byref(prm), _ptr(out2d), cap2d, _ptr(n2d),
                                 _ptr(ncc_out), _ptr(plane_offsets)), h)


def ulm_pair3d(h, t, list2d, n2d, cap2d, n_frames, out3d, cap3d, n3d):
    _check(L.load().ulm_pair3d(h, t, _ptr(list2d), _ptr(n2d), cap2d, n_frames, _ptr(out3d), cap3d, _ptr(n3d)), h)


def make_track_params(length=10, substeps=10, max_step_m=150e-6, max_turn_deg=45.0, max_speed_change=0.5,
                      voxel_m=50e-6) -> L.ulm_track_params:
    import math
    p = L.ulm_track_params()
    p.len, p.substeps, p.max_step_m = length, substeps, max_step_m
    p.cos_max_turn, p.max_speed_change, p.voxel_m = math.cos(math.radians(max_turn_deg)), max_speed_change, voxel_m
    return p


def make_sep_params(prf_hz, n_bands=3, edges_hz=None) -> L.ulm_sep_params:
    """Speed bands of the separation; equal bands over (0, prf / 2] unless
    edges_hz (n_bands + 1 increasing values) is given."""
    if edges_hz is None:
        edges_hz = [i * prf_hz / (2.0 * n_bands) for i in range(n_bands + 1)]
    if len(edges_hz) != n_bands + 1:
        raise ValueError("edges_hz needs n_bands + 1 values")
    p = L.ulm_sep_params()
    p.prf_hz, p.n_bands = prf_hz, n_bands
    for i, e in enumerate(edges_hz):
        p.edges_hz[i] = e
    return p


def ulm_separate(h, t, planes, planes_dtype, n_frames, prm, subsets):
    _check(L.load().ulm_separate(h, t, _ptr(planes), planes_dtype, n_frames, C.byref(prm), _ptr(subsets)), h)


def ulm_separate_enhance(h, t, planes, planes_dtype, n_frames, prm, enh, A, M):
    _check(L.load().ulm_separate_enhance(h, t, _ptr(planes), planes_dtype, n_frames, C.byref(prm), enh, _ptr(A),
                                         _ptr(M)), h)


def rca_clutter_svd(h, t, slices, n_frames, rank, iterations=30):
    _check(L.load().rca_clutter_svd(h, t, _ptr(slices), n_frames, rank, iterations), h)


def rca_clutter_svd_info(h, t, slices, n_frames, rank, iterations, info):
    """info: device float tensor [2K][4] (see rca.h)"""
    _check(L.load().rca_clutter_svd_info(h, t, _ptr(slices), n_frames, rank, iterations, _ptr(info)), h)


def rca_motion_estimate(h, t, slices, n_frames, motion, shifts=None, peaks=None):
    _check(L.load().rca_motion_estimate(h, t, _ptr(slices), n_frames, _ptr(motion), _ptr(shifts), _ptr(peaks)), h)


def ulm_density_shape(t, voxel_m):
    dims = (C.c_int32 * 3)()
    _check(L.load().ulm_density_shape(t, voxel_m, C.cast(dims, C.c_void_p)), None)
    return int(dims[0]), int(dims[1]), int(dims[2])


def ulm_track(h, t, list3d, n3d, cap3d, n_frames, prm, out, cap_tracks, n_tracks, density=None):
    _check(L.load().ulm_track(h, t, _ptr(list3d), _ptr(n3d), cap3d, n_frames, C.byref(prm), _ptr(out), cap_tracks,
                              _ptr(n_tracks), _ptr(density)), h)


def ulm_track_velocity(h, t, tracks, n_tracks, cap_tracks, prm, speed_sum, vz_sum):
    _check(L.load().ulm_track_velocity(h, t, _ptr(tracks), _ptr(n_tracks), cap_tracks, C.byref(prm), _ptr(speed_sum),
                                       _ptr(vz_sum)), h)


def ulm_pair3d_noalloc(h, t, list2d, n2d, cap2d, n_frames, out3d, cap3d, n3d):
    """ulm_pair3d on the library's fixed per-device scratch (no allocation)."""
    _check(L.load().ulm_pair3d_noalloc(h, t, _ptr(list2d), _ptr(n2d), cap2d, n_frames, _ptr(out3d), cap3d, _ptr(n3d)), h)


def ulm_localize(h, t, planes, planes_dtype, n_frames, prm: ulm_params, out2d, cap2d, n2d, out3d, cap3d, n3d):
    _check(L.load().ulm_localize(h, t, _ptr(planes), planes_dtype, n_frames, C.byref(prm), _ptr(out2d), cap2d,
                                 _ptr(n2d), _ptr(out3d), cap3d, _ptr(n3d)), h)


def _batch_items(items):
    arr = (rca_batch_item * len(items))()
    for q, it in enumerate(items):
        a = arr[q]
        a.tables = it["tables"]
        a.rf = _ptr(it["rf"])
        a.scale = _ptr(it.get("scale"))
        a.n_frames = it["n_frames"]
        a.planes = _ptr(it["planes"])
        a.out2d = _ptr(it.get("out2d"))
        a.cap2d = it.get("cap2d", 0)
        a.n2d_dev = _ptr(it.get("n2d"))
        a.out3d = _ptr(it.get("out3d"))
        a.cap3d = it.get("cap3d", 0)
        a.n3d_dev = _ptr(it.get("n3d"))
    return arr


def rca_batch_create(h, items, rf_dtype, iq_dtype, planes_dtype, prm=None):
    """items: sequence of dicts with keys tables, rf, scale, n_frames, planes and
    (with prm) out2d, cap2d, n2d, out3d, cap3d, n3d (tensors or pointers)."""
    arr = _batch_items(items)
    b = C.c_void_p()
    _check(L.load().rca_batch_create(h, len(items), arr, rf_dtype, iq_dtype, planes_dtype,
                                     C.byref(prm) if prm is not None else None, C.byref(b)), h)
    return b


def rca_beamform_projections_batched(h, items, rf_dtype, planes_dtype, prm=None):
    """one-shot batch (plan, one run, synchronise, free); items as rca_batch_create"""
    arr = _batch_items(items)
    _check(L.load().rca_beamform_projections_batched(h, len(items), arr, rf_dtype, planes_dtype,
                                                     C.byref(prm) if prm is not None else None), h)


def rca_batch_run(b, use_graph=False, h=None):
    _check(L.load().rca_batch_run(b, int(bool(use_graph))), h, "rca_batch_run")


def rca_batch_set_mode(b, mode):
    _check(L.load().rca_batch_set_mode(b, int(mode)), None, "rca_batch_set_mode")


def rca_batch_set_wait_limit(b, cycles, block_ensemble=-1):
    _check(L.load().rca_batch_set_wait_limit(b, int(cycles), int(block_ensemble)), None, "rca_batch_set_wait_limit")


def rca_batch_destroy(b):
    _check(L.load().rca_batch_destroy(b), None, "rca_batch_destroy")


def rca_autotune(h, t, iq, iq_dtype, n_frames):
    zt, dc, zp = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(L.load().rca_autotune(h, t, _ptr(iq), iq_dtype, n_frames, C.byref(zt), C.byref(dc), C.byref(zp)), h)
    return zt.value, dc.value, zp.value


def rca_fp32_probe(h, packed, iterations, sink):
    """enqueue the FP32 issue-rate probe; returns the launch's FP32 operations"""
    fl = C.c_double(0.0)
    _check(L.load().rca_fp32_probe(h, int(packed), int(iterations), _ptr(sink), C.byref(fl)), h)
    return fl.value


def ulm_cnn_create(h, channels=32, max_pixels=1 << 22, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0):
    d = ulm_cnn_desc()
    d.channels, d.max_pixels, d.lr, d.beta1, d.beta2, d.eps, d.seed = channels, max_pixels, lr, beta1, beta2, eps, seed
    c = C.c_void_p()
    _check(L.load().ulm_cnn_create(h, C.byref(d), C.byref(c)), h)
    return c


def ulm_cnn_destroy(c):
    _check(L.load().ulm_cnn_destroy(c), None, "ulm_cnn_destroy")


def ulm_cnn_param_count(c) -> int:
    n = C.c_size_t(0)
    _check(L.load().ulm_cnn_param_count(c, C.byref(n)), None, "ulm_cnn_param_count")
    return n.value


def ulm_cnn_set_params(c, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(L.load().ulm_cnn_set_params(c, p.ctypes.data_as(C.c_void_p), p.size), None, "ulm_cnn_set_params")


def ulm_cnn_get_params(c) -> np.ndarray:
    out = np.zeros(ulm_cnn_param_count(c), dtype=np.float32)
    _check(L.load().ulm_cnn_get_params(c, out.ctypes.data_as(C.c_void_p), out.size), None, "ulm_cnn_get_params")
    return out


def ulm_cnn_get_grads(c) -> np.ndarray:
    out = np.zeros(ulm_cnn_param_count(c), dtype=np.float32)
    _check(L.load().ulm_cnn_get_grads(c, out.ctypes.data_as(C.c_void_p), out.size), None, "ulm_cnn_get_grads")
    return out


def ulm_cnn_forward(c, A, M, planes_per_frame, B, H, W, heat):
    _check(L.load().ulm_cnn_forward(c, _ptr(A), _ptr(M), planes_per_frame, B, H, W, _ptr(heat)), None, "ulm_cnn_forward")


def ulm_cnn_infer(c, A, M, planes_per_frame, B, H, W, heat):
    _check(L.load().ulm_cnn_infer(c, _ptr(A), _ptr(M), planes_per_frame, B, H, W, _ptr(heat)), None, "ulm_cnn_infer")


def ulm_cnn_train_step(c, A, M, planes_per_frame, B, H, W, target, loss_dev, apply_update=True):
    _check(L.load().ulm_cnn_train_step(c, _ptr(A), _ptr(M), planes_per_frame, B, H, W, _ptr(target), _ptr(loss_dev),
                                       int(bool(apply_update))), None, "ulm_cnn_train_step")


def ulm_cnn_target(h, pts, n, B, H4, W4, sigma, target):
    _check(L.load().ulm_cnn_target(h, _ptr(pts), n, B, H4, W4, sigma, _ptr(target)), h)


def ulm_cnn_save(c, path: str):
    _check(L.load().ulm_cnn_save(c, path.encode()), None, "ulm_cnn_save")


def ulm_cnn_load(c, path: str):
    _check(L.load().ulm_cnn_load(c, path.encode()), None, "ulm_cnn_load")


def ulm_detect_map(h, t, heat, up, A, M, n_frames, score_min, alpha, out2d, cap2d, n2d):
    _check(L.load().ulm_detect_map(h, t, _ptr(heat), up, _ptr(A), _ptr(M), n_frames, score_min, alpha, _ptr(out2d),
                                   cap2d, _ptr(n2d)), h)
