"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  The CUDA library never does, and
nothing here imports the CUDA library: the two share only the seeded inputs of
``synth``.

The arithmetic lives in ``rca_oracle.c`` (plain loops, double precision,
built with ``-ffp-contract=off``); this module compiles it with gcc on first
use and marshals numpy arrays through ctypes.  Complex arrays are
``complex128`` (interleaved re, im in memory, as the C code expects).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from . import cnn  # noqa: F401  (FP64 CNN reference, same status as this module)


_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "rca_oracle.c")]
_lock = threading.Lock()
_lib = None

MAX_K = 8
FIR_TAPS = 31


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "rca_oracle.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-Wall", *_SRC, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class OrGeom(C.Structure):
    _fields_ = [("n_el", C.c_int), ("nz", C.c_int), ("ns", C.c_int), ("P", C.c_int), ("K", C.c_int),
                ("us", C.c_int),
                ("pitch", C.c_double), ("fc", C.c_double), ("fs", C.c_double), ("c", C.c_double),
                ("z0", C.c_double), ("dz", C.c_double), ("fnum", C.c_double),
                ("ang", C.c_double * (2 * MAX_K))]


LOC2D = np.dtype([("frame", "<i4"), ("axis", "<i4"), ("slab", "<i4"), ("iz", "<i4"), ("ilat", "<i4"),
                  ("z", "<f8"), ("lat", "<f8"), ("ncc", "<f8"), ("amp", "<f8")], align=True)
LOC3D = np.dtype([("frame", "<i4"), ("i_xz", "<i4"), ("i_yz", "<i4"),
                  ("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("amp_xz", "<f8"), ("amp_yz", "<f8")],
                 align=True)

_P = C.c_void_p
_D = C.c_double
_I = C.c_int


class TrackParams(C.Structure):
    _fields_ = [("len", C.c_int), ("substeps", C.c_int), ("max_step", C.c_double), ("cos_max_turn", C.c_double),
                ("max_speed_change", C.c_double), ("voxel", C.c_double)]


TRACK = np.dtype([("first", "<i4"), ("frame0", "<i4"), ("accepted", "<i4"), ("a", "<f8", (3, 3)),
                  ("mean_speed", "<f8"), ("cos_turn", "<f8"), ("speed_range", "<f8")], align=True)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "or_elem_pos": (_D, [_P, _I]),
                "or_depth": (_D, [_P, _I]),
                "or_slice_depth": (_D, [_P, _I]),
                "or_slice_rows": (_I, [_P]),
                "or_t0": (_D, [_P]),
                "or_tau_tx": (_D, [_P, _I, _D, _D]),
                "or_tau_rx": (_D, [_P, _D, _D]),
                "or_apod": (_D, [_P, _D, _D]),
                "or_tau_c": (_D, [_P, _I, _D]),
                "or_shift_dz": (_D, [_P, _I, _D]),
                "or_fir_taps": (None, [_P]),
                "or_demod": (None, [_P, _I, _P, _I, _I, _P, _P]),
                "or_das_volume": (None, [_P, _P, _I, _P]),
                "or_project_volume": (None, [_P, _P, _I, _P]),
                "or_project_direct": (None, [_P, _P, _I, _P]),
                "or_stage1": (None, [_P, _P, _P]),
                "or_stage2_volume": (None, [_P, _P, _I, _P]),
                "or_stage2_project": (None, [_P, _P, _P]),
                "or_xdoppler": (None, [_I, _I, _I, _I, _P, _P, _P]),
                "or_ncc_plane": (None, [_I, _I, _P, _I, _D, _D, _D, _P]),
                "or_peaks_plane": (_I, [_I, _I, _P, _P, _D, _D, _D, _I, _P]),
                "or_localize2d": (_I, [_I, _I, _I, _I, _P, _P, _I, _D, _D, _D, _D, _I, _P]),
                "or_pair3d": (_I, [_I, _P, _I, _I, _P]),
                "or_track_link": (None, [_P, _I, _P, _P, _P, _P, _D, _P]),
                "or_track_build": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _I, _P]),
                "or_track_grid": (None, [_P, _D, _P]),
                "or_track_accumulate": (None, [_P, _I, _P, _P, _P]),
                "or_track_velocity": (None, [_P, _I, _P, _P, _P, _P]),
                "or_set_threads": (None, [_I]),
                "or_max_threads": (_I, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def set_threads(n: int) -> None:
    """OpenMP thread count of the C loops (the CPU baseline's 1-thread and
    all-core timings)."""
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def geom(g) -> OrGeom:
    """C descriptor from a ``synth.RcaGeometry``."""
    if g.K > MAX_K:
        raise ValueError("at most 8 transmissions per family")
    s = OrGeom()
    s.n_el, s.nz, s.ns, s.P, s.K, s.us = g.n_el, g.nz, g.ns, g.P, g.K, g.us
    s.pitch, s.fc, s.fs, s.c, s.z0, s.dz, s.fnum = g.pitch, g.fc, g.fs, g.c, g.z0, g.dz, g.fnum
    for k, a in enumerate(g.angles):
        s.ang[k] = a
    return s


def _byref(s):
    return C.cast(C.pointer(s), C.c_void_p)


# --- geometry definitions ---------------------------------------------------

def tau_tx(g, k, trans, z):
    return lib().or_tau_tx(_byref(geom(g)), k, trans, z)


def tau_rx(g, lat_off, z):
    return lib().or_tau_rx(_byref(geom(g)), lat_off, z)


def apod(g, lat_off, z):
    return lib().or_apod(_byref(geom(g)), lat_off, z)


def tau_c(g, k, z):
    return lib().or_tau_c(_byref(geom(g)), k, z)


def shift_dz(g, k, u):
    return lib().or_shift_dz(_byref(geom(g)), k, u)


def elem_pos(g, e):
    return lib().or_elem_pos(_byref(geom(g)), e)


def depth(g, i):
    return lib().or_depth(_byref(geom(g)), i)


def slice_depth(g, r):
    return lib().or_slice_depth(_byref(geom(g)), r)


def t0(g):
    return lib().or_t0(_byref(geom(g)))


def fir_taps() -> np.ndarray:
    h = np.zeros(FIR_TAPS)
    lib().or_fir_taps(_ptr(h))
    return h


# --- beamforming --------------------------------------------------------------

def demod(g, rf, remove_mean: bool = True, frames=None) -> np.ndarray:
    """rf [F][2K][E][ns] float32 -> IQ complex128 [F'][2K][E][ns] for the listed
    frames (all by default); the mean is taken over all F frames."""
    rf = np.ascontiguousarray(rf, dtype=np.float32)
    F = rf.shape[0]
    assert rf.shape == (F, g.n_tx, g.n_el, g.ns), rf.shape
    if frames is None:
        iq = np.zeros(rf.shape, dtype=np.complex128)
        lib().or_demod(_byref(geom(g)), F, _ptr(rf), int(remove_mean), F, None, _ptr(iq))
    else:
        sel = np.ascontiguousarray(list(frames), dtype=np.int32)
        iq = np.zeros((len(sel),) + rf.shape[1:], dtype=np.complex128)
        lib().or_demod(_byref(geom(g)), F, _ptr(rf), int(remove_mean), len(sel), _ptr(sel), _ptr(iq))
    return iq


def das_volume(g, iq_frame, fam: int) -> np.ndarray:
    """Full 3D DAS of one frame and family -> V [N(x)][N(y)][nz] complex."""
    iq_frame = np.ascontiguousarray(iq_frame, dtype=np.complex128)
    V = np.zeros((g.n_el, g.n_el, g.nz), dtype=np.complex128)
    lib().or_das_volume(_byref(geom(g)), _ptr(iq_frame), fam, _ptr(V))
    return V


def _planes_frame(g):
    return np.zeros((2, 2, g.n_slab, g.nz, g.n_el), dtype=np.complex128)


def project_volume(g, V, fam: int, planes_frame=None) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.complex128)
    out = _planes_frame(g) if planes_frame is None else planes_frame
    lib().or_project_volume(_byref(geom(g)), _ptr(V), fam, _ptr(out))
    return out


def project_direct(g, iq_frame, fam: int, planes_frame=None) -> np.ndarray:
    iq_frame = np.ascontiguousarray(iq_frame, dtype=np.complex128)
    out = _planes_frame(g) if planes_frame is None else planes_frame
    lib().or_project_direct(_byref(geom(g)), _ptr(iq_frame), fam, _ptr(out))
    return out


def stage1(g, iq_frame) -> np.ndarray:
    """Reference slices S [2K][nzs][N] of one frame."""
    iq_frame = np.ascontiguousarray(iq_frame, dtype=np.complex128)
    S = np.zeros((g.n_tx, g.nzs, g.n_el), dtype=np.complex128)
    lib().or_stage1(_byref(geom(g)), _ptr(iq_frame), _ptr(S))
    return S


def stage2_volume(g, S, fam: int) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.complex128)
    V = np.zeros((g.n_el, g.n_el, g.nz), dtype=np.complex128)
    lib().or_stage2_volume(_byref(geom(g)), _ptr(S), fam, _ptr(V))
    return V


def stage2_project(g, S) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.complex128)
    out = _planes_frame(g)
    lib().or_stage2_project(_byref(geom(g)), _ptr(S), _ptr(out))
    return out


def beamform_projections(g, rf, mode: str = "two_stage", remove_mean: bool = True,
                         frames=None, return_slices: bool = False):
    """RF -> projection planes [F'][2][2][S][nz][N] (complex128) for the listed
    frames (all by default).  The mean is always taken over every frame of rf."""
    frames = range(rf.shape[0]) if frames is None else list(frames)
    iq = demod(g, rf, remove_mean, frames)
    planes = np.zeros((len(frames), 2, 2, g.n_slab, g.nz, g.n_el), dtype=np.complex128)
    slices = np.zeros((len(frames), g.n_tx, g.nzs, g.n_el), dtype=np.complex128) if return_slices else None
    for q in range(len(frames)):
        if mode == "two_stage":
            S = stage1(g, iq[q])
            if slices is not None:
                slices[q] = S
            planes[q] = stage2_project(g, S)
        elif mode == "direct":
            project_direct(g, iq[q], 0, planes[q])
            project_direct(g, iq[q], 1, planes[q])
        elif mode == "volume":
            for fam in (0, 1):
                project_volume(g, das_volume(g, iq[q], fam), fam, planes[q])
        else:
            raise ValueError(mode)
    return (planes, slices) if return_slices else planes


# --- localisation ---------------------------------------------------------------

def xdoppler(planes) -> tuple:
    """planes [F][2][2][S][nz][N] -> (A [F][2][S][nz][N], M [F])."""
    planes = np.ascontiguousarray(planes, dtype=np.complex128)
    F, _, _, S, nz, N = planes.shape
    A = np.zeros((F, 2, S, nz, N))
    M = np.zeros(F)
    lib().or_xdoppler(F, S, nz, N, _ptr(planes), _ptr(A), _ptr(M))
    return A, M


def ncc_plane(A2, d: int, sig_z: float, sig_l: float, Mt: float) -> np.ndarray:
    A2 = np.ascontiguousarray(A2, dtype=np.float64)
    out = np.zeros_like(A2)
    lib().or_ncc_plane(A2.shape[0], A2.shape[1], _ptr(A2), d, sig_z, sig_l, Mt, _ptr(out))
    return out


def peaks_plane(A2, ncc, Mt, alpha, ncc_min, cap: int = 1 << 16) -> np.ndarray:
    A2 = np.ascontiguousarray(A2, dtype=np.float64)
    ncc = np.ascontiguousarray(ncc, dtype=np.float64)
    out = np.zeros(cap, dtype=LOC2D)
    n = lib().or_peaks_plane(A2.shape[0], A2.shape[1], _ptr(A2), _ptr(ncc), Mt, alpha, ncc_min,
                             cap, _ptr(out))
    return out[:min(n, cap)]


def localize2d(A, M, d, sig_z, sig_l, alpha, ncc_min, cap: int = 1 << 20) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    F, _, S, nz, N = A.shape
    out = np.zeros(cap, dtype=LOC2D)
    n = lib().or_localize2d(F, S, nz, N, _ptr(A), _ptr(M), d, sig_z, sig_l, alpha, ncc_min,
                            cap, _ptr(out))
    if n > cap:
        raise RuntimeError(f"oracle 2D list capacity {cap} < {n}")
    return out[:n]


def pair3d(list2d, P: int, cap: int = 1 << 20) -> np.ndarray:
    L = np.ascontiguousarray(list2d, dtype=LOC2D)
    out = np.zeros(cap, dtype=LOC3D)
    n = lib().or_pair3d(len(L), _ptr(L) if len(L) else None, P, cap, _ptr(out))
    if n > cap:
        raise RuntimeError(f"oracle 3D list capacity {cap} < {n}")
    return out[:n]


def localize(planes, d, sig_z, sig_l, alpha, ncc_min, P):
    """planes -> (A, M, list2d, list3d)."""
    A, M = xdoppler(planes)
    L2 = localize2d(A, M, d, sig_z, sig_l, alpha, ncc_min)
    L3 = pair3d(L2, P)
    return A, M, L2, L3


# --- tracking (Sec. II-A6) ----------------------------------------------------------

def track_params(length=10, substeps=10, max_step=150e-6, max_turn_deg=45.0, max_speed_change=0.5,
                 voxel=50e-6) -> TrackParams:
    import math
    return TrackParams(length, substeps, max_step, math.cos(math.radians(max_turn_deg)), max_speed_change, voxel)


def _list_columns(list3d):
    L = np.ascontiguousarray(list3d)
    return (np.ascontiguousarray(L["frame"], dtype=np.int32), np.ascontiguousarray(L["x"], dtype=np.float64),
            np.ascontiguousarray(L["y"], dtype=np.float64), np.ascontiguousarray(L["z"], dtype=np.float64))


def track_link(g, list3d, max_step: float) -> np.ndarray:
    """successor of each 3D localisation in the next frame (-1: none); the list is frame-major"""
    fr, x, y, z = _list_columns(list3d)
    succ = np.full(len(fr), -1, dtype=np.int32)
    lib().or_track_link(_byref(geom(g)), len(fr), _ptr(fr), _ptr(x), _ptr(y), _ptr(z), max_step, _ptr(succ))
    return succ


def track_build(g, list3d, succ, prm: TrackParams, cap: int = 1 << 20) -> np.ndarray:
    fr, x, y, z = _list_columns(list3d)
    succ = np.ascontiguousarray(succ, dtype=np.int32)
    out = np.zeros(cap, dtype=TRACK)
    n = lib().or_track_build(_byref(geom(g)), len(fr), _ptr(fr), _ptr(x), _ptr(y), _ptr(z), _ptr(succ),
                             _byref(prm), cap, _ptr(out))
    if n > cap:
        raise RuntimeError(f"oracle track capacity {cap} < {n}")
    return out[:n]


def track_grid(g, voxel: float) -> tuple:
    dims = np.zeros(3, dtype=np.int32)
    lib().or_track_grid(_byref(geom(g)), voxel, _ptr(dims))
    return int(dims[0]), int(dims[1]), int(dims[2])


def track_accumulate(g, tracks, prm: TrackParams) -> np.ndarray:
    """density counts [nz_v][ny_v][nx_v] (uint32)"""
    nx, ny, nz = track_grid(g, prm.voxel)
    grid = np.zeros((nz, ny, nx), dtype=np.uint32)
    tr = np.ascontiguousarray(tracks, dtype=TRACK)
    lib().or_track_accumulate(_byref(geom(g)), len(tr), _ptr(tr) if len(tr) else None, _byref(prm), _ptr(grid))
    return grid


def track_velocity(g, tracks, prm: TrackParams):
    """velocity sums (speed, axial component) per voxel [nz_v][ny_v][nx_v] (int64,
    nanometres per frame interval, one term per accumulation sample)"""
    nx, ny, nz = track_grid(g, prm.voxel)
    speed = np.zeros((nz, ny, nx), dtype=np.int64)
    vz = np.zeros((nz, ny, nx), dtype=np.int64)
    tr = np.ascontiguousarray(tracks, dtype=TRACK)
    lib().or_track_velocity(_byref(geom(g)), len(tr), _ptr(tr) if len(tr) else None, _byref(prm), _ptr(speed),
                            _ptr(vz))
    return speed, vz


def track(g, list3d, prm: TrackParams):
    """list3d -> (successors, tracks, density counts)"""
    succ = track_link(g, list3d, prm.max_step)
    tr = track_build(g, list3d, succ, prm)
    return succ, tr, track_accumulate(g, tr, prm)
