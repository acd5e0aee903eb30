"""ctypes declarations of librca (include/rca.h).  Loading fails loudly if the
library has not been built: there is no fallback implementation."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librca.so")
# RCA_LIBRARY=checked selects the bounds-checked build (see build.py)
LIB_CHECKED_PATH = os.path.join(HERE, "_build", "librca_checked.so")

RCA_MAX_K = 8
ULM_PAIR3D_NOALLOC_MAX_2D = 1 << 19
ULM_PAIR3D_NOALLOC_MAX_PLANES = 1 << 16

# rca_status
RCA_OK = 0
RCA_ERR_INVALID_ARG = 1
RCA_ERR_SHAPE = 2
RCA_ERR_UNSUPPORTED = 3
RCA_ERR_CUDA = 4
RCA_ERR_CAPACITY = 5
RCA_ERR_TIMEOUT = 6
RCA_ERR_BOUNDS = 7

# rca_dtype
RCA_F32, RCA_I16, RCA_F16, RCA_C32, RCA_C16F, RCA_C16BF = range(6)

RCA_MODE_TWO_STAGE, RCA_MODE_DIRECT = 0, 1
RCA_BATCH_PERSISTENT, RCA_BATCH_STAGED = 0, 1
RCA_CLUTTER_NONE, RCA_CLUTTER_MEAN, RCA_CLUTTER_SVD = 0, 1, 2
ULM_ENH_XDOPPLER, ULM_ENH_COHERENT = 0, 1

(RCA_TAB_TX_F64, RCA_TAB_RX_F64, RCA_TAB_TX_Q16, RCA_TAB_RX_Q16, RCA_TAB_W, RCA_TAB_DMAX,
 RCA_TAB_S2_SHIFT, RCA_TAB_S2_PSI, RCA_TAB_S2_EC, RCA_TAB_S2_COEF, RCA_TAB_S2_TMIN) = range(11)


class rca_geometry_desc(C.Structure):
    _fields_ = [("n_el", C.c_int), ("nz", C.c_int), ("ns", C.c_int), ("P", C.c_int), ("K", C.c_int),
                ("us", C.c_int),
                ("pitch_m", C.c_double), ("fc_hz", C.c_double), ("fs_hz", C.c_double),
                ("c_mps", C.c_double), ("z0_m", C.c_double), ("dz_m", C.c_double), ("fnum", C.c_double),
                ("ang_rc_rad", C.POINTER(C.c_double)), ("ang_cr_rad", C.POINTER(C.c_double))]


class rca_bf_params(C.Structure):
    _fields_ = [("mode", C.c_int), ("clutter", C.c_int), ("iq_dtype", C.c_int), ("svd_rank", C.c_int),
                ("svd_iterations", C.c_int), ("reserved", C.c_int * 3)]


class ulm_params(C.Structure):
    _fields_ = [("d", C.c_int), ("sig_z", C.c_float), ("sig_lat", C.c_float), ("alpha", C.c_float),
                ("ncc_min", C.c_float), ("enh", C.c_int), ("reserved", C.c_int * 4)]


class rca_batch_item(C.Structure):
    _fields_ = [("tables", C.c_void_p), ("rf", C.c_void_p), ("scale", C.c_void_p), ("n_frames", C.c_int),
                ("planes", C.c_void_p), ("out2d", C.c_void_p), ("cap2d", C.c_int), ("n2d_dev", C.c_void_p),
                ("out3d", C.c_void_p), ("cap3d", C.c_int), ("n3d_dev", C.c_void_p)]


class ulm_cnn_desc(C.Structure):
    _fields_ = [("channels", C.c_int), ("max_pixels", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_ulonglong)]


class ulm_track_params(C.Structure):
    _fields_ = [("len", C.c_int32), ("substeps", C.c_int32), ("max_step_m", C.c_double), ("cos_max_turn", C.c_double),
                ("max_speed_change", C.c_double), ("voxel_m", C.c_double)]


ULM_TRACK_MAX_LEN = 64
ULM_SEP_MAX_BANDS = 4


class ulm_sep_params(C.Structure):
    _fields_ = [("prf_hz", C.c_double), ("n_bands", C.c_int32), ("reserved", C.c_int32),
                ("edges_hz", C.c_double * (ULM_SEP_MAX_BANDS + 1))]
TRACK = np.dtype([("first", "<i4"), ("frame0", "<i4"), ("accepted", "<i4"), ("reserved", "<i4"),
                  ("a", "<f8", (3, 3)), ("mean_speed", "<f8"), ("cos_turn", "<f8"), ("speed_range", "<f8")])
assert TRACK.itemsize == 112

LOC2D = np.dtype([("frame", "<i4"), ("axis", "<i4"), ("slab", "<i4"), ("iz", "<i4"), ("ilat", "<i4"),
                  ("z", "<f4"), ("lat", "<f4"), ("ncc", "<f4"), ("amp", "<f4"), ("reserved", "<i4")])
LOC3D = np.dtype([("frame", "<i4"), ("i_xz", "<i4"), ("i_yz", "<i4"), ("reserved", "<i4"),
                  ("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("amp_xz", "<f4"), ("amp_yz", "<f4"),
                  ("reserved2", "<f4")])
assert LOC2D.itemsize == 40 and LOC3D.itemsize == 40

_P = C.c_void_p
_I = C.c_int
_S = C.c_int  # rca_status
_SZ = C.c_size_t

# name -> (restype, argtypes); every symbol declared in include/rca.h
SIGNATURES = {
    "rca_version": (_I, []),
    "rca_status_string": (C.c_char_p, [_S]),
    "rca_create": (_S, [C.POINTER(_P), _I]),
    "rca_destroy": (_S, [_P]),
    "rca_set_stream": (_S, [_P, _P]),
    "rca_last_error": (C.c_char_p, [_P]),
    "rca_sync_status": (_S, [_P, C.POINTER(_I)]),
    "rca_reserve": (_S, [_P, _P, _I]),
    "rca_geometry_create": (_S, [_P, C.POINTER(rca_geometry_desc), C.POINTER(_P)]),
    "rca_geometry_destroy": (_S, [_P]),
    "rca_delay_tables": (_S, [_P, _P, C.POINTER(_P)]),
    "rca_tables_destroy": (_S, [_P]),
    "rca_tables_query": (_S, [_P, _I, C.POINTER(_SZ), C.POINTER(_I)]),
    "rca_tables_download": (_S, [_P, _I, _P, _SZ]),
    "rca_ingest": (_S, [_P, _P, _P, _I, _P, _I, _I, _P, _I]),
    "rca_stage1": (_S, [_P, _P, _P, _I, _I, _P]),
    "rca_stage2_project": (_S, [_P, _P, _P, _I, _P, _I]),
    "rca_direct_project": (_S, [_P, _P, _P, _I, _I, _P, _I]),
    "rca_beamform_projections": (_S, [_P, _P, _P, _I, _P, _I, C.POINTER(rca_bf_params), _P, _I]),
    "ulm_enhance": (_S, [_P, _P, _P, _I, _I, _I, _P, _P]),
    "ulm_detect2d": (_S, [_P, _P, _P, _P, _I, C.POINTER(ulm_params), _P, _I, _P, _P, _P]),
    "ulm_pair3d": (_S, [_P, _P, _P, _P, _I, _I, _P, _I, _P]),
    "ulm_pair3d_noalloc": (_S, [_P, _P, _P, _P, _I, _I, _P, _I, _P]),
    "ulm_localize": (_S, [_P, _P, _P, _I, _I, C.POINTER(ulm_params), _P, _I, _P, _P, _I, _P]),
    "ulm_density_shape": (_S, [_P, C.c_double, _P]),
    "rca_motion_estimate": (_S, [_P, _P, _P, _I, _P, _P, _P]),
    "rca_clutter_svd": (_S, [_P, _P, _P, _I, _I, _I]),
    "rca_clutter_svd_info": (_S, [_P, _P, _P, _I, _I, _I, _P]),
    "ulm_separate": (_S, [_P, _P, _P, _I, _I, C.POINTER(ulm_sep_params), _P]),
    "ulm_separate_enhance": (_S, [_P, _P, _P, _I, _I, C.POINTER(ulm_sep_params), _I, _P, _P]),
    "ulm_track": (_S, [_P, _P, _P, _P, _I, _I, C.POINTER(ulm_track_params), _P, _I, _P, _P]),
    "ulm_track_velocity": (_S, [_P, _P, _P, _P, _I, C.POINTER(ulm_track_params), _P, _P]),
    "ulm_cnn_create": (_S, [_P, C.POINTER(ulm_cnn_desc), C.POINTER(_P)]),
    "ulm_cnn_destroy": (_S, [_P]),
    "ulm_cnn_param_count": (_S, [_P, C.POINTER(_SZ)]),
    "ulm_cnn_set_params": (_S, [_P, _P, _SZ]),
    "ulm_cnn_get_params": (_S, [_P, _P, _SZ]),
    "ulm_cnn_get_grads": (_S, [_P, _P, _SZ]),
    "ulm_cnn_forward": (_S, [_P, _P, _P, _I, _I, _I, _I, _P]),
    "ulm_cnn_infer": (_S, [_P, _P, _P, _I, _I, _I, _I, _P]),
    "ulm_cnn_train_step": (_S, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _I]),
    "ulm_cnn_target": (_S, [_P, _P, _I, _I, _I, _I, C.c_float, _P]),
    "ulm_cnn_save": (_S, [_P, C.c_char_p]),
    "ulm_cnn_load": (_S, [_P, C.c_char_p]),
    "ulm_detect_map": (_S, [_P, _P, _P, _I, _P, _P, _I, C.c_float, C.c_float, _P, _I, _P]),
    "rca_batch_create": (_S, [_P, _I, C.POINTER(rca_batch_item), _I, _I, _I, C.POINTER(ulm_params), C.POINTER(_P)]),
    "rca_beamform_projections_batched": (_S, [_P, _I, C.POINTER(rca_batch_item), _I, _I, C.POINTER(ulm_params)]),
    "rca_batch_run": (_S, [_P, _I]),
    "rca_batch_set_mode": (_S, [_P, _I]),
    "rca_batch_set_wait_limit": (_S, [_P, C.c_longlong, _I]),
    "rca_batch_destroy": (_S, [_P]),
    "rca_autotune": (_S, [_P, _P, _P, _I, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "rca_fp32_probe": (_S, [_P, _I, _I, _P, C.POINTER(C.c_double)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = None):
    """Load librca.so (librca_checked.so when RCA_LIBRARY=checked) and declare
    every entry point.  Raises if missing."""
    global _lib
    with _lock:
        if _lib is None:
            if path is None:
                path = LIB_CHECKED_PATH if os.environ.get("RCA_LIBRARY") == "checked" else LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"librca not built ({path} missing); run `python -m paper_2511_21647_gb300.build`")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib
