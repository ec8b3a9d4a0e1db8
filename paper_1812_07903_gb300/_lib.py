"""ctypes declarations of the C ABI in include/slso.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslso.so")

SLSO_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "DTYPE", 4: "OOM", 5: "CUDA",
    6: "NONFINITE", 7: "TIMEOUT", 8: "BUSY", 9: "NOT_FOUND", 10: "CANCELLED",
}
F64, F32, BF16, FP8_E4M3 = 0, 1, 2, 3
COUNTSKETCH, SRHT, GAUSSIAN, OSNAP = 0, 1, 2, 3
KIND = {"countsketch": COUNTSKETCH, "srht": SRHT, "gaussian": GAUSSIAN, "osnap": OSNAP}
POLICY = {"dec": 0, "swr": 1, "swor": 2}
DTYPE = {"f64": F64, "f32": F32, "bf16": BF16, "fp8": FP8_E4M3}

# Every symbol include/slso.h declares.
EXPORTS = (
    "slso_version", "slso_last_error", "slso_create", "slso_destroy", "slso_workspace_size",
    "slso_sketch", "slso_sketched_svd", "slso_gram", "slso_leverage", "slso_order", "slso_rank_rows_host",
    "slso_profile", "slso_profile_read", "slso_order_static", "slso_sample_order",
    "slso_rank_rows_host_batch", "slso_set_pool_limit", "slso_set_score_form", "slso_selftest_wait", "slso_server_cancel",
    "slso_approx_u", "slso_rank_rows_streamed",
    "slso_server_create", "slso_server_destroy", "slso_server_submit", "slso_server_poll", "slso_server_stats",
    "slso_server_counters",
)
JOB_LEVERAGE, JOB_SKETCHED_SVD = 0, 1
STAGES = ("sketch", "qr", "solve", "scores", "order", "copy", "syrk", "chol")


class Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("compute", ctypes.c_int32), ("s", ctypes.c_int64),
        ("k", ctypes.c_int64), ("seed_S", ctypes.c_uint64), ("seed_Pi", ctypes.c_uint64),
        ("tau", ctypes.c_double), ("correct_frac", ctypes.c_double), ("nnz", ctypes.c_int32),
        ("factor", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("rank", ctypes.c_int64), ("sigma_max", ctypes.c_double), ("sigma_min_kept", ctypes.c_double),
        ("score_sum", ctypes.c_double), ("tau", ctypes.c_double), ("nonfinite", ctypes.c_int32),
        ("svd_route", ctypes.c_int32), ("svd_sweeps", ctypes.c_int32), ("gram_route", ctypes.c_int32),
        ("gram_resid", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Job(ctypes.Structure):
    _fields_ = [
        ("job", ctypes.c_int32), ("xdt", ctypes.c_int32), ("X", ctypes.c_void_p),
        ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("ldx", ctypes.c_int64), ("params", Params),
        ("scores", ctypes.c_void_p), ("order", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
        ("V", ctypes.c_void_p), ("R", ctypes.c_void_p),
    ]


class SlsoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"slso {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load():
    """Load libslso.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1812_07903_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "slso_version": ([], ctypes.c_char_p),
        "slso_last_error": ([], ctypes.c_char_p),
        "slso_create": ([ctypes.POINTER(vp), ctypes.c_int], i32),
        "slso_destroy": ([vp], i32),
        "slso_workspace_size": ([ctypes.POINTER(Params), i64, i64, ctypes.POINTER(ctypes.c_size_t)], i32),
        "slso_sketch": ([vp, vp, i64, i64, i64, i32, i32, i64, u64, vp, vp], i32),
        "slso_sketched_svd": ([vp, vp, i64, i64, dbl, vp, vp, vp, ctypes.POINTER(Info), vp], i32),
        "slso_gram": ([vp, vp, i64, i64, vp, vp], i32),
        "slso_leverage": ([vp, vp, i64, i64, i64, i32, ctypes.POINTER(Params), vp, ctypes.POINTER(Info), vp], i32),
        "slso_order": ([vp, vp, i32, i64, vp, vp], i32),
        "slso_rank_rows_host": ([vp, vp, i64, i64, i64, i32, ctypes.POINTER(Params), vp, vp,
                                 ctypes.POINTER(Info), vp], i32),
        "slso_order_static": ([vp, i32, i64, vp, vp], i32),
        "slso_sample_order": ([vp, vp, i32, i64, i32, ctypes.c_uint64, vp, vp], i32),
        "slso_rank_rows_host_batch": ([vp, i64, vp, i64, i64, i64, i32, vp, vp, vp, vp, vp], i32),
        "slso_set_pool_limit": ([vp, ctypes.c_size_t], i32),
        "slso_set_score_form": ([vp, i32], i32),
        "slso_rank_rows_streamed": ([vp, vp, i64, i64, i64, i32, ctypes.POINTER(Params), i64, vp, vp,
                                     ctypes.POINTER(Info), vp], i32),
        "slso_approx_u": ([vp, vp, i64, i64, i64, i32, ctypes.POINTER(Params), vp, i64, ctypes.POINTER(Info), vp], i32),
        "slso_selftest_wait": ([vp, i32, i64, vp], i32),
        "slso_server_cancel": ([vp, i64], i32),
        "slso_server_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_size_t], i32),
        "slso_server_destroy": ([vp], i32),
        "slso_server_counters": ([vp, ctypes.POINTER(i64), i32], i32),
        "slso_server_submit": ([vp, ctypes.POINTER(Job), ctypes.POINTER(i64)], i32),
        "slso_server_poll": ([vp, i64, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(Info),
                              ctypes.POINTER(ctypes.c_double)], i32),
        "slso_server_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t)], i32),
        "slso_profile": ([vp, ctypes.c_int], i32),
        "slso_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status):
    if status != SLSO_OK:
        raise SlsoError(status, load().slso_last_error().decode())
