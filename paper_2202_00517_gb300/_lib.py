"""ctypes binding of libknnd.so (include/knnd.h): same names, argument
marshalling only.  Loading fails loudly when the library has not been built;
there is no fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libknnd.so")

KNND_OK = 0
KNND_EINVAL = -1
KNND_EDOMAIN = -2
KNND_ENOMEM = -3
KNND_ECUDA = -4
KNND_ETIMEOUT = -5
KNND_EOVERFLOW = -6
KNND_ESTATE = -7

KNND_F32 = 0
KNND_F64 = 1
KNND_PREC_FP64 = 0
KNND_PREC_MIXED_FP32 = 1
KNND_PREC_MIXED_BF16X3 = 2
KNND_PREC_AUTO = 3

KNND_MAX_K = 64
KNND_MAX_M = 128
KNND_MAX_ROUNDS = 64

KNND_STOP_FCC = 1
KNND_STOP_ZERO = 2
KNND_STOP_MAX_ROUNDS = 3
KNND_STOP_DELTA = 4
KNND_CMP_KL = 0
KNND_CMP_KL_REVERSE = 1
KNND_CMP_SQEUCLIDEAN = 2
KNND_CMP_INNER = 3
KNND_LOOP_AUTO = 0
KNND_LOOP_HOST = 1
KNND_LOOP_GRAPH = 2
KNND_JOIN_TMA = 1
KNND_JOIN_PLAIN = 2
KNND_JOIN_FP64 = 3
KNND_JOIN_TC = 4

EXPORTS = [
    "knnd_create", "knnd_destroy", "knnd_set_stream", "knnd_prepare", "knnd_init_graph", "knnd_round",
    "knnd_fcc", "knnd_sync", "knnd_build", "knnd_build_host", "knnd_get_stats", "knnd_reset_stats",
    "knnd_status_string", "knnd_version", "knnd_fcc_noalloc", "knnd_batch_create", "knnd_batch_run",
    "knnd_batch_info", "knnd_batch_destroy", "knnd_build_batched", "knnd_philox4x32_10",
    "knnd_fma_peak",
]

KNND_NOALLOC_MAX_SAMPLES = 1 << 20


class knnd_params(ctypes.Structure):
    _fields_ = [("fcc_samples", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("stop_on_zero_updates", ctypes.c_int32), ("debug", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("incremental", ctypes.c_int32), ("stop_delta", ctypes.c_float),
                ("comparator", ctypes.c_int32), ("loop", ctypes.c_int32), ("split_den", ctypes.c_int32),
                ("merge_keep", ctypes.c_int32), ("join_blocks", ctypes.c_int32), ("join_form", ctypes.c_int32)]


class knnd_build_info(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("updates", ctypes.c_int64 * KNND_MAX_ROUNDS),
                ("fcc_hits", ctypes.c_int64 * (KNND_MAX_ROUNDS + 1)),
                ("proposals", ctypes.c_int64), ("init_pairs", ctypes.c_int64),
                ("rescored", ctypes.c_int64), ("bound_violations", ctypes.c_int64),
                ("merge_fallbacks", ctypes.c_int64), ("join_survivors", ctypes.c_int64),
                ("bound_audited", ctypes.c_int64), ("join_kernel", ctypes.c_int32), ("reserved", ctypes.c_int32)]


KNND_NUM_PHASES = 6
PHASES = ("prepare", "init", "csr", "join", "merge", "fcc")


class knnd_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64),
                ("phase_count", ctypes.c_int64 * KNND_NUM_PHASES),
                ("phase_ms", ctypes.c_double * KNND_NUM_PHASES)]


class knnd_instance(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("ld", ctypes.c_int64), ("n", ctypes.c_int64),
                ("m", ctypes.c_int32), ("K", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("idx", ctypes.c_void_p), ("key", ctypes.c_void_p)]


class KnndError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libknnd.so (raises when it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing")
    lib = ctypes.CDLL(path)
    P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    sig = {
        "knnd_create": (i32, [ctypes.POINTER(P), i64, i32, i32, i32, i32, ctypes.POINTER(knnd_params), P]),
        "knnd_destroy": (None, [P]),
        "knnd_set_stream": (i32, [P, P]),
        "knnd_prepare": (i32, [P, P, i64]),
        "knnd_init_graph": (i32, [P, P, i64, u64, P, P, P]),
        "knnd_round": (i32, [P, P, i64, u64, i32, P, P, P, P, P]),
        "knnd_fcc": (i32, [P, P, u64, i32, P]),
        "knnd_sync": (i32, [P]),
        "knnd_build": (i32, [P, P, i64, u64, P, P, P, ctypes.POINTER(knnd_build_info)]),
        "knnd_build_host": (i32, [P, P, i64, u64, P, P, ctypes.POINTER(knnd_build_info)]),
        "knnd_get_stats": (i32, [P, ctypes.POINTER(knnd_stats)]),
        "knnd_reset_stats": (i32, [P]),
        "knnd_status_string": (ctypes.c_char_p, [i32]),
        "knnd_version": (i32, []),
        "knnd_fcc_noalloc": (i32, [P, i64, i32, u64, i32, i32, P, P]),
        "knnd_batch_create": (i32, [ctypes.POINTER(P), i32, P, i32, i32, ctypes.POINTER(knnd_params), i64, P]),
        "knnd_batch_run": (i32, [P, P]),
        "knnd_batch_info": (i32, [P, P, P, P]),
        "knnd_batch_destroy": (None, [P]),
        "knnd_build_batched": (i32, [i32, P, i32, i32, ctypes.POINTER(knnd_params), i64, P, P]),
        "knnd_philox4x32_10": (i32, [P, P, i64, P]),
        "knnd_fma_peak": (i32, [i32, i32, i64, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().knnd_status_string(status).decode()


def check(status: int, where: str) -> None:
    if status != KNND_OK:
        raise KnndError(status, where)
