"""ctypes binding of libetdrdpif (include/etdrdpif.h): argument marshalling only.

Every function keeps its C name.  The library must have been built in-tree
(``python -m paper_2001_11220_gb300.build`` or ``__graft_entry__.build()``);
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libetdrdpif.so")

ETD_OK, ETD_ERR_INVALID_ARG, ETD_ERR_UNSUPPORTED, ETD_ERR_OOM, ETD_ERR_CUDA, ETD_ERR_TIMEOUT, ETD_ERR_NONFINITE = range(7)
STATUS_NAMES = {0: "ETD_OK", 1: "ETD_ERR_INVALID_ARG", 2: "ETD_ERR_UNSUPPORTED", 3: "ETD_ERR_OOM",
                4: "ETD_ERR_CUDA", 5: "ETD_ERR_TIMEOUT", 6: "ETD_ERR_NONFINITE"}
ETD_FP64, ETD_FP32 = 0, 1

# every symbol include/etdrdpif.h declares
EXPORTS = ["etd_create", "etd_create_coupled", "etd_step", "etd_run", "etd_run_host", "etd_step_adjoint", "etd_grad", "etd_run_vjp",
           "etd_batch_create", "etd_batch_run", "etd_batch_autotune", "etd_batch_set_wait_limit",
           "etd_batch_debug_hold", "etd_check_finite", "etd_autotune", "etd_set_stream", "etd_profile",
           "etd_profile_read", "etd_get_info", "etd_step_noalloc",
           "etd_last_error", "etd_destroy"]


class etd_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("bc", ctypes.c_int32 * 3), ("n", ctypes.c_int64 * 3),
                ("length", ctypes.c_double * 3)]


class etd_reaction(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nspecies", ctypes.c_int32), ("params", ctypes.c_double * 8)]


class etd_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nspecies", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("npoints", ctypes.c_int64), ("state_bytes", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_int64), ("launches_per_step", ctypes.c_int32),
                ("chunk", ctypes.c_int32 * 3), ("lines_per_block", ctypes.c_int32 * 3),
                ("staged", ctypes.c_int32 * 3), ("pack", ctypes.c_int32 * 3), ("grid_blocks", ctypes.c_int32 * 3)]


class EtdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2001_11220_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    dptr = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "etd_create": ([ctypes.POINTER(etd_grid), dptr, ctypes.POINTER(etd_reaction), dbl, i32, vp, pp], i32),
        "etd_create_coupled": ([ctypes.POINTER(etd_grid), dptr, ctypes.POINTER(etd_reaction), dbl, i32, vp, pp],
                               i32),
        "etd_step": ([vp, vp, dbl], i32),
        "etd_check_finite": ([vp, vp, ctypes.POINTER(i64)], i32),
        "etd_run": ([vp, vp, dbl, i64], i32),
        "etd_run_host": ([vp, vp, dbl, i64], i32),
        "etd_step_adjoint": ([vp, vp, dbl, vp, vp, dptr, dptr], i32),
        "etd_grad": ([vp, vp, dbl, vp, i64, i64, dptr, vp, dptr, dptr], i32),
        "etd_run_vjp": ([vp, vp, dbl, i64, i64, vp, vp, dptr, dptr], i32),
        "etd_batch_create": ([i32, ctypes.POINTER(etd_grid), dptr, ctypes.POINTER(etd_reaction), dbl, i32, vp, pp], i32),
        "etd_batch_run": ([vp, pp, dbl, i64], i32),
        "etd_batch_autotune": ([vp, pp], i32),
        "etd_batch_set_wait_limit": ([vp, dbl], i32),
        "etd_batch_debug_hold": ([vp, i32, i32], i32),
        "etd_autotune": ([vp, vp], i32),
        "etd_set_stream": ([vp, vp], i32),
        "etd_profile": ([vp, i32], i32),
        "etd_profile_read": ([vp, dptr, ctypes.POINTER(ctypes.c_int64)], i32),
        "etd_get_info": ([vp, ctypes.POINTER(etd_info)], i32),
        "etd_step_noalloc": ([ctypes.POINTER(etd_grid), dptr, ctypes.POINTER(etd_reaction), dbl, i32, vp, dbl, vp], i32),
        "etd_last_error": ([vp], ctypes.c_char_p),
        "etd_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status: int, ctx=None):
    if status != ETD_OK:
        msg = load().etd_last_error(ctx)
        raise EtdError(status, msg.decode() if msg else "")
