"""Torch-side convenience around the librca binding: one handle, geometry and
table set per session, output buffers allocated with torch on the handle's
device, work enqueued on torch's current stream.  No computation happens
here; every step is a librca call."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from . import rca as R

_TORCH_COMPLEX = {
    L.RCA_C32: (torch.float32, 2),
    L.RCA_C16F: (torch.float16, 2),
    L.RCA_C16BF: (torch.bfloat16, 2),
}


def complex_buffer(shape, dtype_code: int, device) -> torch.Tensor:
    """Interleaved complex buffer [..., 2] of the given librca complex dtype."""
    tdt, two = _TORCH_COMPLEX[dtype_code]
    return torch.empty((*shape, two), dtype=tdt, device=device)


class RcaSession:
    def __init__(self, geom, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("librca needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.geom = geom
        torch.cuda.set_device(self.device)
        self.h = R.rca_create(device)
        R.rca_set_stream(self.h, torch.cuda.current_stream(self.device))
        self.g = R.rca_geometry_create(self.h, geom)
        self.t = R.rca_delay_tables(self.h, self.g)
        self.S = geom.n_el // geom.P

    # -- shapes -------------------------------------------------------------
    def planes_shape(self, F):
        g = self.geom
        return (F, 2, 2, self.S, g.nz, g.n_el)

    def a_shape(self, F):
        g = self.geom
        return (F, 2, self.S, g.nz, g.n_el)

    def slices_shape(self, F):
        g = self.geom
        return (F, 2 * len(g.ang_rc), (g.nz - 1) * g.us + 1, g.n_el)

    def iq_shape(self, F):
        g = self.geom
        return (F, 2 * len(g.ang_rc), g.ns, g.n_el)

    # -- steps ----------------------------------------------------------------
    def bind_stream(self, stream=None):
        R.rca_set_stream(self.h, stream or torch.cuda.current_stream(self.device))

    def ingest(self, rf, rf_dtype=L.RCA_F32, scale=None, clutter=L.RCA_CLUTTER_MEAN, iq_dtype=L.RCA_C32):
        F = rf.shape[0]
        iq = complex_buffer(self.iq_shape(F), iq_dtype, self.device)
        R.rca_ingest(self.h, self.t, rf, rf_dtype, scale, F, clutter, iq, iq_dtype)
        return iq

    def stage1(self, iq, iq_dtype=L.RCA_C32):
        F = iq.shape[0]
        sl = complex_buffer(self.slices_shape(F), L.RCA_C32, self.device)
        R.rca_stage1(self.h, self.t, iq, iq_dtype, F, sl)
        return sl

    def stage2(self, slices, planes_dtype=L.RCA_C32):
        F = slices.shape[0]
        pl = complex_buffer(self.planes_shape(F), planes_dtype, self.device)
        R.rca_stage2_project(self.h, self.t, slices, F, pl, planes_dtype)
        return pl

    def direct(self, iq, iq_dtype=L.RCA_C32, planes_dtype=L.RCA_C32):
        F = iq.shape[0]
        pl = complex_buffer(self.planes_shape(F), planes_dtype, self.device)
        R.rca_direct_project(self.h, self.t, iq, iq_dtype, F, pl, planes_dtype)
        return pl

    def beamform(self, rf, rf_dtype=L.RCA_F32, scale=None, mode=L.RCA_MODE_TWO_STAGE,
                 clutter=L.RCA_CLUTTER_MEAN, iq_dtype=L.RCA_C32, planes_dtype=L.RCA_C32, out=None, svd_rank=0,
                 svd_iterations=0):
        F = rf.shape[0]
        pl = out if out is not None else complex_buffer(self.planes_shape(F), planes_dtype, self.device)
        R.rca_beamform_projections(self.h, self.t, rf, rf_dtype, scale, F,
                                   R.bf_params(mode, clutter, iq_dtype, svd_rank, svd_iterations), pl, planes_dtype)
        return pl

    def enhance(self, planes, planes_dtype=L.RCA_C32, enh=L.ULM_ENH_XDOPPLER):
        F = planes.shape[0]
        A = torch.empty(self.a_shape(F), dtype=torch.float32, device=self.device)
        M = torch.empty(F, dtype=torch.float32, device=self.device)
        R.ulm_enhance(self.h, self.t, planes, planes_dtype, F, enh, A, M)
        return A, M

    def separate(self, planes, prm, planes_dtype=L.RCA_C32):
        """complex subsets [2 nb][F][2][2][S][nz][N] (Sec. II-A5)"""
        F = planes.shape[0]
        out = torch.empty((2 * prm.n_bands,) + tuple(self.planes_shape(F)) + (2,), dtype=torch.float32,
                          device=self.device)
        R.ulm_separate(self.h, self.t, planes, planes_dtype, F, prm, out)
        return out

    def separate_enhance(self, planes, prm, planes_dtype=L.RCA_C32, enh=L.ULM_ENH_XDOPPLER):
        """per-subset amplitude A [2 nb][F][2][S][nz][N] and maxima M [2 nb][F]"""
        F = planes.shape[0]
        ns = 2 * prm.n_bands
        A = torch.empty((ns,) + tuple(self.a_shape(F)), dtype=torch.float32, device=self.device)
        M = torch.empty((ns, F), dtype=torch.float32, device=self.device)
        R.ulm_separate_enhance(self.h, self.t, planes, planes_dtype, F, prm, enh, A, M)
        return A, M

    def detect2d(self, A, M, prm, cap2d=1 << 16, want_ncc=False):
        F = A.shape[0]
        out = torch.zeros((max(cap2d, 1), 10), dtype=torch.int32, device=self.device)
        n2d = torch.zeros(1, dtype=torch.int32, device=self.device)
        ncc = torch.zeros_like(A) if want_ncc else None
        R.ulm_detect2d(self.h, self.t, A, M, F, prm, out, cap2d, n2d, ncc)
        return out, n2d, ncc

    def pair3d(self, list2d_dev, n2d_dev, cap2d, F, cap3d=1 << 16):
        out = torch.zeros((max(cap3d, 1), 10), dtype=torch.int32, device=self.device)
        n3d = torch.zeros(1, dtype=torch.int32, device=self.device)
        R.ulm_pair3d(self.h, self.t, list2d_dev, n2d_dev, cap2d, F, out, cap3d, n3d)
        return out, n3d

    def localize(self, planes, prm, planes_dtype=L.RCA_C32, cap2d=1 << 16, cap3d=1 << 16, bufs=None):
        F = planes.shape[0]
        if bufs is None:
            bufs = self.loc_buffers(cap2d, cap3d)
        out2d, n2d, out3d, n3d = bufs
        R.ulm_localize(self.h, self.t, planes, planes_dtype, F, prm, out2d, cap2d, n2d, out3d, cap3d, n3d)
        return bufs

    def loc_buffers(self, cap2d, cap3d):
        return (torch.zeros((max(cap2d, 1), 10), dtype=torch.int32, device=self.device),
                torch.zeros(1, dtype=torch.int32, device=self.device),
                torch.zeros((max(cap3d, 1), 10), dtype=torch.int32, device=self.device),
                torch.zeros(1, dtype=torch.int32, device=self.device))

    def sync_status(self) -> int:
        return R.rca_sync_status(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            R.rca_tables_destroy(self.t)
            R.rca_geometry_destroy(self.g)
            R.rca_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def list2d_numpy(buf: torch.Tensor, n: int) -> np.ndarray:
    """Device 2D-list buffer -> structured numpy array of its first n entries."""
    raw = buf[:n].contiguous().cpu().numpy()
    return raw.view(L.LOC2D).reshape(-1)


def list3d_numpy(buf: torch.Tensor, n: int) -> np.ndarray:
    raw = buf[:n].contiguous().cpu().numpy()
    return raw.view(L.LOC3D).reshape(-1)


def to_complex128(t: torch.Tensor) -> np.ndarray:
    """[..., 2] interleaved (any float dtype) -> numpy complex128."""
    a = t.float().cpu().numpy()
    return a[..., 0].astype(np.float64) + 1j * a[..., 1].astype(np.float64)
