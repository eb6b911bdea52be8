"""ctypes binding of libcvrpsd.so (include/cvrpsd.h). Argument marshalling
only: every step of the Split runs in the library's CUDA kernels. Importing
this module never falls back to anything: if the library is missing it raises."""
from __future__ import annotations

import ctypes
import os
import platform

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", platform.machine(), "libcvrpsd.so")

OK = 0
WARN_INFEASIBLE = 1
ERR_ARG = -1
ERR_DTYPE = -2
ERR_OVERFLOW = -3
ERR_CUDA = -4
ERR_DEVICE_STATUS = -5
ERR_NOMEM = -6
ERR_UNSUPPORTED = -7
ERR_TIMEOUT = -8
I16 = 2
I32 = 4
MAX_N = 8191
KERNEL_AUTO, KERNEL_DEQUE, KERNEL_WARP, KERNEL_SEQPAR = 0, 1, 2, 3
GEN_NORMAL, GEN_CORRELATED = 0, 1
WALK_AUTO, WALK_GLOBAL_TABLE, WALK_PARAM_TABLE = 0, 1, 2

# Every symbol include/cvrpsd.h declares.
EXPORTS = [
    "cvrpsd_create", "cvrpsd_destroy", "cvrpsd_strerror", "cvrpsd_last_error",
    "cvrpsd_version", "cvrpsd_set_config", "cvrpsd_get_config", "cvrpsd_last_stats",
    "cvrpsd_split_eval", "cvrpsd_split_eval_host", "cvrpsd_gen_demand", "cvrpsd_set_profiling", "cvrpsd_debug_fail_alloc",
    "cvrpsd_check_inputs", "cvrpsd_set_log", "cvrpsd_split_eval_noalloc", "cvrpsd_batch_create", "cvrpsd_batch_run", "cvrpsd_batch_results",
    "cvrpsd_batch_destroy", "cvrpsd_batch_autotune", "cvrpsd_split_eval_batch", "cvrpsd_autotune", "cvrpsd_split_routes",
    "cvrpsd_split_eval_tours", "cvrpsd_neighbors", "cvrpsd_topk", "cvrpsd_gather_tours", "cvrpsd_accept_best",
    "cvrpsd_surrogate_create", "cvrpsd_surrogate_destroy", "cvrpsd_surrogate_predict",
    "cvrpsd_surrogate_train_step", "cvrpsd_surrogate_gradients", "cvrpsd_surrogate_params", "cvrpsd_surrogate_state",
    "cvrpsd_surrogate_set_scale", "cvrpsd_int_rate",
]
SURROGATE_PARAMS = 67841
NOALLOC_MAX_S = 1048576


# void (*)(int32_t level, const char *message, void *user)
LOG_FN = ctypes.CFUNCTYPE(None, ctypes.c_int32, ctypes.c_char_p, ctypes.c_void_p)
LOG_ERROR, LOG_INFO, LOG_DEBUG = 0, 1, 2


class Config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("spt", ctypes.c_int32), ("ring", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("rounds", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("spt", ctypes.c_int32), ("ring", ctypes.c_int32),
                ("overflow", ctypes.c_int64), ("launches", ctypes.c_int32),
                ("kernel_ms", ctypes.c_float), ("fallback_ms", ctypes.c_float),
                ("variant", ctypes.c_int32), ("rounds", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best", Config), ("best_ms", ctypes.c_float), ("best_dtype", ctypes.c_int32),
                ("shapes_timed", ctypes.c_int32)]


class TourDesc(ctypes.Structure):
    _fields_ = [("tour", ctypes.c_void_p), ("n", ctypes.c_int32), ("dist", ctypes.c_void_p),
                ("demand", ctypes.c_void_p), ("ld", ctypes.c_int64), ("Q", ctypes.c_int32),
                ("L", ctypes.c_int32), ("out_cost", ctypes.c_void_p)]


class CvrpsdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the library (built by `build.build()`); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libcvrpsd.so not built at {p}: run paper_2511_18022_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.cvrpsd_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.cvrpsd_destroy.argtypes = [vp]
    lib.cvrpsd_strerror.argtypes = [ctypes.c_int]
    lib.cvrpsd_strerror.restype = ctypes.c_char_p
    lib.cvrpsd_last_error.argtypes = [vp]
    lib.cvrpsd_last_error.restype = ctypes.c_char_p
    lib.cvrpsd_version.restype = ctypes.c_char_p
    lib.cvrpsd_set_config.argtypes = [vp, ctypes.POINTER(Config)]
    lib.cvrpsd_get_config.argtypes = [vp, ctypes.POINTER(Config)]
    lib.cvrpsd_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.cvrpsd_set_profiling.argtypes = [vp, i32]
    lib.cvrpsd_debug_fail_alloc.argtypes = [vp, ctypes.c_int32]
    lib.cvrpsd_check_inputs.argtypes = [vp, vp]
    lib.cvrpsd_set_log.argtypes = [vp, LOG_FN, vp, i32]
    lib.cvrpsd_int_rate.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.cvrpsd_split_eval.argtypes = [vp, vp, i32, vp, vp, i32, i64, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.cvrpsd_split_eval_host.argtypes = [vp, vp, i32, vp, vp, i32, i64, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.cvrpsd_gen_demand.argtypes = [vp, ctypes.c_uint64, i32, vp, vp, i32, i64, i64, i32, vp, vp]
    lib.cvrpsd_split_eval_noalloc.argtypes = [vp, i32, vp, vp, i32, i64, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.cvrpsd_split_routes.argtypes = [vp, vp, i32, vp, vp, i32, i64, i64, i32, i32, vp, vp, i64, vp, vp,
                                        vp, vp]
    lib.cvrpsd_split_eval_tours.argtypes = [vp, vp, i32, i32, vp, vp, i32, i64, i64, i32, i32, vp, vp, vp, vp]
    lib.cvrpsd_neighbors.argtypes = [vp, vp, i32, vp, i32, vp, vp]
    lib.cvrpsd_topk.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.cvrpsd_gather_tours.argtypes = [vp, vp, i32, i32, vp, i32, vp, vp]
    lib.cvrpsd_accept_best.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
    lib.cvrpsd_surrogate_create.argtypes = [vp, i32, vp, vp, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.cvrpsd_surrogate_destroy.argtypes = [vp]
    lib.cvrpsd_surrogate_predict.argtypes = [vp, vp, i32, vp, vp]
    lib.cvrpsd_surrogate_train_step.argtypes = [vp, vp, i32, vp, ctypes.c_float, vp, vp]
    lib.cvrpsd_surrogate_gradients.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.cvrpsd_surrogate_params.argtypes = [vp, vp, vp, ctypes.POINTER(i64)]
    lib.cvrpsd_surrogate_state.argtypes = [vp, vp, vp, ctypes.POINTER(i64)]
    lib.cvrpsd_surrogate_set_scale.argtypes = [vp, ctypes.c_float, ctypes.c_float]
    lib.cvrpsd_autotune.argtypes = [vp, vp, i32, vp, vp, i32, i64, i64, i32, i32, ctypes.c_char_p,
                                    ctypes.POINTER(TuneResult), vp]
    lib.cvrpsd_batch_create.argtypes = [vp, i32, ctypes.POINTER(TourDesc), i64, i32, ctypes.POINTER(vp)]
    lib.cvrpsd_batch_run.argtypes = [vp, vp]
    lib.cvrpsd_batch_results.argtypes = [vp, vp, vp, vp, vp]
    lib.cvrpsd_batch_destroy.argtypes = [vp]
    lib.cvrpsd_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(TourDesc), i64, i32, ctypes.POINTER(TuneResult), vp]
    lib.cvrpsd_split_eval_batch.argtypes = [vp, i32, ctypes.POINTER(TourDesc), i64, i32, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        getattr(lib, name)          # raises AttributeError if a symbol is missing
    if path is None:
        _lib = lib
    return lib


def check(ctx, rc: int, allow_warn: bool = True) -> int:
    if rc < 0 or (rc > 0 and not allow_warn):
        lib = load()
        detail = lib.cvrpsd_last_error(ctx).decode() if ctx else ""
        raise CvrpsdError(rc, f"{lib.cvrpsd_strerror(rc).decode()}: {detail}")
    return rc
