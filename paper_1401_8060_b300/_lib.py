"""ctypes declarations of libstk.so (the C ABI in include/stk.h).

The library must exist: there is no fallback.  A missing or unloadable
libstk.so raises at first use with the path that was tried.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# STK_LIBRARY selects another build of the same ABI (the bounds-checked
# libstk_debug.so); by default the release library beside this file.
LIB_PATH = os.environ.get("STK_LIBRARY") or os.path.join(HERE, "libstk.so")

STK_OK, STK_EINVAL, STK_ENOMEM, STK_ECUDA, STK_ETIMEOUT, STK_ESTATE, STK_ECANCELED = 0, -1, -2, -3, -4, -5, -6
STK_EBOUNDS = -7
STK_BATCH_MAX_K = 32
STK_HOST_PTR, STK_SIGMA_PER_FREQ, STK_NORM_PAPER, STK_FP16 = 0x1, 0x2, 0x4, 0x8
STK_OUT_HOST = 0x1
STK_MAX_K = 4096
STK_NOALLOC_MAX_TRACKS = 1 << 20
STK_OPT_KERNEL, STK_OPT_THREADS, STK_OPT_MAX_R, STK_OPT_STAGES, STK_OPT_SMEM_KB = 1, 2, 3, 4, 5
STK_OPT_WAIT_MS, STK_OPT_WITHHOLD_SLAB, STK_OPT_ORDER, STK_OPT_SELECT_SAMPLE = 6, 7, 8, 9
STK_OPT_INTERP_THREADS = 10

# Every entry point declared in include/stk.h: (name, restype, argtypes).
_vp = C.c_void_p
SIGNATURES = [
    ("stk_version", C.c_int, []),
    ("stk_build_flags", C.c_int, []),
    ("stk_create", C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
    ("stk_destroy", None, [_vp]),
    ("stk_set_stream", C.c_int, [_vp, _vp]),
    ("stk_load_map", C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint,
                               C.POINTER(_vp)]),
    ("stk_update_map", C.c_int, [_vp, _vp, _vp, _vp, C.c_uint]),
    ("stk_free_map", None, [_vp]),
    ("stk_map_info", C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_uint)]),
    ("stk_set_tracks", C.c_int, [_vp, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double]),
    ("stk_score", C.c_int, [_vp, _vp, C.c_int, _vp, C.c_uint]),
    ("stk_score_all", C.c_int, [_vp, _vp, _vp]),
    ("stk_track_params", C.c_int, [_vp, _vp, C.c_uint64, _vp, C.POINTER(C.c_double), _vp]),
    ("stk_score_explicit", C.c_int, [_vp, _vp, _vp, _vp, C.c_uint64, _vp]),
    ("stk_sync", C.c_int, [_vp]),
    ("stk_set_profiling", C.c_int, [_vp, C.c_int]),
    ("stk_last_timings", C.c_int, [_vp, C.POINTER(C.c_double)]),
    ("stk_set_option", C.c_int, [_vp, C.c_int, C.c_int64]),
    ("stk_last_plan", C.c_int, [_vp, C.POINTER(C.c_int64)]),
    ("stk_last_error", C.c_char_p, [_vp]),
    ("stk_set_template_shape", C.c_int, [_vp, C.c_int, C.c_int]),
    ("stk_set_tau_prior", C.c_int, [_vp, _vp, C.c_int]),
    ("stk_track_times", C.c_int, [_vp, _vp, C.c_uint64, _vp]),
    ("stk_score_explicit_general", C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint64, _vp]),
    ("stk_interp_forward", C.c_int, [_vp, _vp, _vp, _vp, C.c_uint64, _vp]),
    ("stk_interp_adjoint", C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint64, _vp, _vp]),
    ("stk_refine", C.c_int, [_vp, _vp, _vp, _vp, C.c_uint64, C.c_int, C.c_float, C.c_float, C.c_float, _vp]),
    ("stk_polish", C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_uint64, C.c_double, C.c_int, _vp, _vp]),
    ("stk_batch_create", C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp, C.c_double, C.POINTER(_vp)]),
    ("stk_batch_destroy", None, [_vp]),
    ("stk_batch_score", C.c_int, [_vp, C.c_int, _vp, C.c_uint]),
    ("stk_batch_cancel", C.c_int, [_vp, C.c_int]),
    ("stk_batch_tune", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int64)]),
    ("stk_score_noalloc", C.c_int, [_vp, C.c_uint64, C.c_uint64, C.c_uint64, C.c_double, C.c_int, _vp, _vp,
                                    _vp]),
]

HIT_DTYPE = np.dtype([("snr", "<f8"), ("index", "<u8"), ("f", "<u4", (3,)), ("reserved", "<u4"),
                      ("tau", "<f8")])
assert HIT_DTYPE.itemsize == 40

_lib = None


def lib():
    """Load libstk.so once and declare its entry points."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libstk.so not found at {LIB_PATH}; build it with "
                "`python -m paper_1401_8060_b300.build` (nvcc, sm_103a). There is no CPU fallback.")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
