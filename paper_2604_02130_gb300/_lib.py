"""ctypes declarations of the C ABI in include/fd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfd.so")

FD_OK = 0
FD_ERR_INVALID = -1
FD_ERR_UNSUPPORTED = -2
FD_ERR_CUDA = -3
FD_ERR_NUMERIC = -4
FD_ERR_TIMEOUT = -5
FD_ERR_TOO_LARGE = -6
FD_NOALLOC_MAX_BATCH = 64
FD_NOALLOC_MAX_NX = 72

FD_PREC_FP64 = 0
FD_PREC_MIXED_TF32 = 1
FD_PREC_MIXED_3XTF32 = 2
PRECISIONS = {"fp64": FD_PREC_FP64, "tf32": FD_PREC_MIXED_TF32, "3xtf32": FD_PREC_MIXED_3XTF32}

FD_WANT_LOGDET = 1
FD_WANT_GREEN = 2
FD_WANT_FORCE = 4

FD_NX_MAX = 288


class fd_problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("nt", ctypes.c_int32),
        ("n_stab", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("expA", ctypes.c_void_p),
        ("expA_inv", ctypes.c_void_p),
        ("phi", ctypes.c_void_p),
    ]


class fd_bss_slice(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("G", ctypes.c_void_p),
        ("phi_row", ctypes.c_void_p),
        ("dphi", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("accepted", ctypes.c_void_p),
    ]


class fd_sparse_hop(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int32),
        ("nfac", ctypes.c_int32),
        ("col", ctypes.c_void_p),
        ("val", ctypes.c_void_p),
    ]


# (name, restype, argtypes) of every exported function of include/fd.h
_VP = ctypes.c_void_p
_I = ctypes.c_int
_PP = ctypes.POINTER(fd_problem)
SIGNATURES = [
    ("fd_ctx_create", _I, [ctypes.POINTER(_VP), _I]),
    ("fd_ctx_destroy", None, [_VP]),
    ("fd_last_error", ctypes.c_char_p, [_VP]),
    ("fd_reserve", _I, [_VP, _I, _PP, _I, _I]),
    ("fd_logdet", _I, [_VP, _I, _PP, _VP, _I, _VP]),
    ("fd_green", _I, [_VP, _I, _PP, _VP, _VP, _I, _VP]),
    ("fd_force", _I, [_VP, _I, _PP, _VP, _VP, _VP, _I, _VP]),
    ("fd_green_tau", _I, [_VP, _I, _PP, _VP, _VP, _VP, _VP, _I, _VP]),
    ("fd_observables", _I, [_VP, _I, _PP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP]),
    ("fd_bss_update", _I, [_VP, _I, ctypes.POINTER(fd_bss_slice), _VP, _VP]),
    ("fd_green_sparse", _I, [_VP, _I, ctypes.POINTER(fd_problem), ctypes.POINTER(fd_sparse_hop),
                             _VP, ctypes.POINTER(_VP), _VP]),
    ("fd_taylor_factors", _I, [_I, ctypes.POINTER(ctypes.c_double)]),
    ("fd_debug_skip_chains", _I, [_VP, _I]),
    ("fd_set_force_split", _I, [_VP, _I]),
    ("fd_status", _I, [_VP, _VP, ctypes.POINTER(_I), _I]),
    ("fd_last_launch_count", _I, [_VP]),
    ("fd_measure_fp64_peak", _I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    ("fd_measure_fp64_issue", _I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    ("fd_check_fp64_refinements", _I, [_VP, _VP, _VP, _I, _VP, _VP]),
    ("fd_set_timing", _I, [_VP, _I]),
    ("fd_last_kernel_ms", _I, [_VP, ctypes.POINTER(ctypes.c_double), _I]),
    ("fd_logdet_noalloc", _I, [_I, _PP, _VP, _VP, _VP, _VP]),
    ("fd_plan_query", _I, [_VP, _I, _PP, _I, _I, ctypes.POINTER(_I), _I]),
    ("fd_graph_create", _I, [_VP, _I, _PP, _VP, _VP, _VP, _I, ctypes.POINTER(_VP)]),
    ("fd_graph_launch", _I, [_VP, _VP, _VP]),
    ("fd_graph_destroy", _I, [_VP, _VP]),
    ("fd_tune", _I, [_VP, _I, _PP, _I, _I, _I]),
    ("fd_tune_nstab", _I, [_VP, _PP, ctypes.POINTER(_I), _I, ctypes.c_double, _I,
                           ctypes.POINTER(_I)]),
    ("fd_tune_nstab_stats", _I, [_VP, _PP, ctypes.POINTER(_I), _I, ctypes.c_double, _I,
                                 ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]),
    ("fd_tune_save", _I, [_VP, ctypes.c_char_p]),
    ("fd_tune_load", _I, [_VP, ctypes.c_char_p]),
]

_lib = None


def load(path: str | None = None):
    """Load libfd.so (building it first if it is missing).  Raises if that is impossible:
    there is no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        from . import build as _build

        _build.build()
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
