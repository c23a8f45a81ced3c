"""ctypes binding of libdfgks.so (the C ABI of include/dfgks.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  If the library is missing the import
of this module succeeds but the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdfgks.so")

OK, EINVAL, ENOMEM, ECUDA, ENONPHYS, ENONPOS, ENAN, ETIMEOUT, ENOTSUP = range(9)


class Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc_xlo", C.c_int), ("bc_xhi", C.c_int), ("bc_ylo", C.c_int), ("bc_yhi", C.c_int),
                ("alpha_thres", C.c_double), ("dH", C.c_double), ("dL", C.c_double), ("eps", C.c_double),
                ("C1", C.c_double), ("C2", C.c_double),
                ("time_limiter", C.c_int), ("tau_reading", C.c_int), ("gp_fallback", C.c_int),
                ("time_scheme", C.c_int), ("dt_rule", C.c_int), ("df_states", C.c_int),
                ("alpha_source", C.c_int)]


class Counters(C.Structure):
    _fields_ = [("fallbacks", C.c_ulonglong), ("df_normal", C.c_ulonglong), ("df_tangential", C.c_ulonglong)]


class BlockPlan(C.Structure):
    _fields_ = [("i0", C.c_int), ("i1", C.c_int), ("j0", C.c_int), ("j1", C.c_int),
                ("bc", C.c_int * 4), ("neighbour", C.c_int * 4)]


class HaloWindow(C.Structure):
    _fields_ = [("neighbour", C.c_int), ("di", C.c_int), ("dj", C.c_int), ("si", C.c_int), ("sj", C.c_int),
                ("w", C.c_int), ("h", C.c_int)]


BC_EXTERNAL = 3      # a block side whose ghost layers a halo copy fills


class DfgksError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, status_string(status), status))


_lock = threading.Lock()
_lib = None
_D = C.POINTER(C.c_double)
_V = C.c_void_p

# name -> argtypes (restype int unless noted)
SIGNATURES = {
    "dfgks_config_default": [C.POINTER(Config), C.c_int, C.c_int],
    "dfgks_create": [C.POINTER(Config), _V, C.POINTER(_V)],
    "dfgks_destroy": [_V],
    "dfgks_set_ic": [_V, _V, C.c_int],
    "dfgks_get_state": [_V, _V, _V, _D, C.POINTER(C.c_long), C.c_int],
    "dfgks_set_state": [_V, _V, _V, C.c_double, C.c_long, C.c_int],
    "dfgks_step": [_V, C.c_int, C.c_double, C.c_int, C.c_double, _D, C.POINTER(C.c_int)],
    "dfgks_residual": [_V, _V, _V, C.c_double, C.c_int, _V, _V, _V, _V],
    "dfgks_adjoint_residual": [_V, _V, _V, C.c_double, C.c_int, _V, _V, _V, _V],
    "dfgks_face_records": [_V, _V, _V, C.c_double, C.c_int, C.c_int, _V],
    "dfgks_get_counters": [_V, C.POINTER(Counters)],
    "dfgks_last_error_detail": [_V, C.POINTER(C.c_long), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "dfgks_device_bytes": [_V, C.POINTER(C.c_ulonglong)],
    "dfgks_set_timing": [_V, C.c_int],
    "dfgks_get_timing": [_V, _V, _V, _V, C.c_int],
    "dfgks_probe_fp64": [C.c_int, _D, _D],
    "dfgks_residual_noalloc": [C.POINTER(Config), _V, _V, _V, C.c_double, C.c_int, _V, _V, _V, _V],
    "dfgks_batch_create": [_V, _V, C.c_int, _V, C.POINTER(_V)],
    "dfgks_batch_destroy": [_V],
    "dfgks_batch_set_ic": [_V, C.c_int, _V, C.c_int],
    "dfgks_batch_step": [_V, C.c_int, C.c_int],
    "dfgks_batch_get_state": [_V, C.c_int, _V, _V, _D, C.POINTER(C.c_long), C.c_int],
    "dfgks_batch_status": [_V, C.c_int, C.POINTER(C.c_long), C.POINTER(C.c_int), C.POINTER(C.c_ulonglong)],
    "dfgks_batch_set_blocks": [_V, _V],
    "dfgks_batch_prepare": [_V, C.c_int],
    "dfgks_batch_autotune": [_V, _V, _D],
    "dfgks_adjoint_steps": [_V, _V, C.c_int, _D, C.c_int, C.c_int, _V, _V],
    "dfgks_forward_checkpointed": [_V, _V, C.c_int, _D, C.c_int, C.c_int, _D],
    "dfgks_adjoint_checkpointed": [_V, _V, _V],
    "dfgks_decomp_plan": [C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.POINTER(BlockPlan)],
    "dfgks_decomp_halo": [C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(HaloWindow)],
    "dfgks_decomp_create": [C.POINTER(Config), C.c_int, C.c_int, _V, C.POINTER(_V)],
    "dfgks_decomp_destroy": [_V],
    "dfgks_decomp_set_ic": [_V, _V, C.c_int],
    "dfgks_decomp_step": [_V, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)],
    "dfgks_decomp_get_state": [_V, _V, _V, _D, C.POINTER(C.c_long), C.c_int],
    "dfgks_decomp_status": [_V, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(Counters)],
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libdfgks.so is not built (run `python -c \"import __graft_entry__ as g; g.build()\"`); "
                                   "there is no CPU fallback")
            L = C.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.dfgks_status_string.argtypes = [C.c_int]
            L.dfgks_status_string.restype = C.c_char_p
            _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().dfgks_status_string(int(status)).decode()
    except Exception:
        return "status %d" % status


def check(rc: int, where: str) -> None:
    if rc != OK:
        raise DfgksError(rc, where)


def exported_symbols() -> list:
    return sorted(list(SIGNATURES) + ["dfgks_status_string"])
