"""ctypes declarations of libmc.so (include/mc.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libmc.so")

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ENOTCONVERGED = 0, 1, 2, 3, 4
MC_EBUSY, MC_PENDING, MC_ETIMEOUT, MC_ECANCELLED, MC_EINTERNAL = 5, 6, 7, 8, 9


class McParams(C.Structure):
    _fields_ = [("tau", C.c_double), ("delta", C.c_double), ("eps", C.c_double), ("l", C.c_int), ("s", C.c_int),
                ("p0", C.c_int), ("p_min", C.c_int), ("p_max", C.c_int), ("i_max", C.c_int), ("i_reuse", C.c_int),
                ("q_reuse", C.c_int), ("recycle", C.c_int), ("k_max", C.c_int), ("precision", C.c_int),
                ("inner", C.c_int), ("seed", C.c_uint64)]


class McIterInfo(C.Structure):
    _fields_ = [("i", C.c_int), ("k", C.c_int), ("r", C.c_int), ("p", C.c_int), ("nsvd", C.c_int),
                ("recycled", C.c_int), ("converged", C.c_int), ("reserved", C.c_int), ("err", C.c_double),
                ("sigma_last", C.c_double), ("sigma_max", C.c_double), ("c", C.c_double), ("norm2", C.c_double)]


class McTiming(C.Structure):
    _fields_ = [("ms", C.c_double), ("bytes", C.c_double), ("flops", C.c_double), ("launches", C.c_int64)]


TIMING_NAMES = ["spmm", "spmm_t", "gram", "gemm", "small", "eig", "sddmm", "other"]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class McAllocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class McJobDesc(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("params", McParams)]


class McResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("r", C.c_int), ("converged", C.c_int),
                ("err", C.c_double), ("m", C.c_int64), ("n", C.c_int64), ("Us", C.POINTER(C.c_float)),
                ("V", C.POINTER(C.c_float)), ("sigma", C.POINTER(C.c_float)), ("queue_s", C.c_double),
                ("latency_s", C.c_double), ("footprint_bytes", C.c_size_t), ("device_bytes_peak", C.c_size_t),
                ("message", C.c_char_p)]


class McServerInfo(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("in_use_bytes", C.c_size_t), ("peak_in_use_bytes", C.c_size_t),
                ("active", C.c_int), ("peak_active", C.c_int), ("queued", C.c_int), ("slots", C.c_int),
                ("admitted", C.c_int64), ("completed", C.c_int64)]


_P = C.c_void_p
_SIGS = {
    "mc_params_default": (None, [C.POINTER(McParams)]),
    "mc_last_error": (C.c_char_p, []),
    "mc_launch_count": (C.c_int64, []),
    "mc_status_str": (C.c_char_p, [C.c_int]),
    "mc_create": (C.c_int, [C.POINTER(_P), C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, _P, C.POINTER(McAllocator)]),
    "mc_create_coo": (C.c_int, [C.POINTER(_P), C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, _P, C.POINTER(McAllocator)]),
    "mc_destroy": (None, [_P]),
    "mc_set_values": (C.c_int, [_P, _P]),
    "mc_get_values": (C.c_int, [_P, _P]),
    "mc_rsvd_bki": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, _P, _P, _P, C.POINTER(C.c_int)]),
    "mc_rsvd_pi": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, _P, _P, _P, C.POINTER(C.c_int)]),
    "mc_rsvd_basic": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, _P, _P, _P, C.POINTER(C.c_int)]),
    "mc_set_precision": (C.c_int, [_P, C.c_int]),
    "mc_svt_step": (C.c_int, [_P, C.POINTER(McParams), C.POINTER(McIterInfo)]),
    "mc_svt_reset": (C.c_int, [_P]),
    "mc_svt_solve": (C.c_int, [_P, C.POINTER(McParams), C.POINTER(McIterInfo)]),
    "mc_svt_factors": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(C.c_int)]),
    "mc_svt_sample": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "mc_timing_enable": (C.c_int, [_P, C.c_int]),
    "mc_timing_read": (C.c_int, [_P, C.POINTER(McTiming)]),
    "mc_omega": (C.c_int, [C.c_int64, C.c_int, C.c_uint64, C.c_uint64, C.c_int, _P, _P]),
    "mc_spmm": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "mc_eig_sym": (C.c_int, [C.c_int, C.c_int, _P, _P, _P]),
    "mc_gram": (C.c_int, [C.c_int64, C.c_int, _P, _P]),
    "mc_join": (C.c_int, [_P]),
    "mc_orth_block": (C.c_int, [C.c_int64, C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, _P, C.c_int, _P]),
    "mc_gram_tc": (C.c_int, [C.c_int64, C.c_int, _P, _P]),
    "mc_panel_gemm": (C.c_int, [C.c_int64, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "mc_gather_rate": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "mc_panel_gram": (C.c_int, [C.c_int64, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "mc_gram_noalloc": (C.c_int, [C.c_int64, C.c_int, _P, C.c_int, _P, C.c_int, _P]),
    "mc_server_create": (C.c_int, [C.POINTER(_P), C.c_size_t, C.c_int, C.c_int, C.c_int]),
    "mc_server_destroy": (None, [_P]),
    "mc_submit": (C.c_int, [_P, C.POINTER(McJobDesc), C.POINTER(C.c_uint64)]),
    "mc_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(McResult)]),
    "mc_wait": (C.c_int, [_P, C.c_uint64, C.c_double]),
    "mc_cancel": (C.c_int, [_P, C.c_uint64]),
    "mc_result_release": (C.c_int, [_P, C.c_uint64]),
    "mc_server_stats": (C.c_int, [_P, C.POINTER(McServerInfo)]),
    "mc_server_admit_order": (C.c_int64, [_P, C.POINTER(C.c_uint64), C.c_int64]),
}

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libmc.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libmc.so not built ({_LIB_PATH}); run `python -m paper_1810_06860_gb300.build`")
    lib = C.CDLL(_LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)
