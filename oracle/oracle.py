"""ctypes wrapper of the plain C oracle (oracle.c).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may use this module.  It shares
no code with the CUDA library; see the header of oracle.c for the readings of
arXiv:2202.00517 it implements (KL comparator of Sec. 2.2, pool and update of
Sec. 3.1 / Sec. 4.2, initial K-out graph of Sec. 3.2, friend clustering rate
and stop rule of Sec. 3.3, brute-force K-NN of Sec. 2.3, diameter of Sec. 3.2
and Sec. 4.3).

All floating-point work is IEEE binary64.  Points are passed as float64 arrays
(float32 inputs are widened exactly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build_oracle", "philox4x32_10", "stream_words", "bounded_draws", "logs", "keys_pairs",
    "init_graph", "round_", "pools", "indegree", "fcc", "build", "bruteforce",
    "diameter_exact", "diameter_bounds", "num_threads",
]


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        sig = {
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_stream_words": (None, [u64, u32, u32, u32, i64, P]),
            "orc_bounded_draws": (None, [u64, u32, u32, u32, u32, i64, P]),
            "orc_logs": (None, [P, i64, ctypes.c_int, P, P]),
            "orc_keys_pairs": (None, [P, i64, ctypes.c_int, P, P, i64, P]),
            "orc_init_graph": (None, [P, i64, ctypes.c_int, ctypes.c_int, u64, P, P]),
            "orc_round": (i64, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, i64, P, P, P, P]),
            "orc_pools": (None, [P, i64, ctypes.c_int, i64, i64, P, P]),
            "orc_indegree": (None, [P, i64, ctypes.c_int, P]),
            "orc_fcc": (i64, [P, i64, ctypes.c_int, u64, i32, i32]),
            "orc_set_comparator": (None, [i32]),
            "orc_build": (i32, [P, i64, ctypes.c_int, ctypes.c_int, u64, i32, i32, i32, ctypes.c_double,
                                P, P, P, P, P]),
            "orc_bruteforce": (None, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P]),
            "orc_diameter_exact": (i32, [P, i64, ctypes.c_int]),
            "orc_diameter_bounds": (None, [P, i64, ctypes.c_int, i32, u64, P, P]),
            "orc_num_threads": (i32, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


_dir_lock = threading.Lock()


COMPARATORS = {"kl": 0, "kl_reverse": 1, "sqeuclidean": 2, "inner": 3}


class _comparator:
    """Comparator for the calls inside: "kl" ranks y for x by D(x||y) (the
    paper's), "kl_reverse" by D(y||x), "sqeuclidean" by |x - y|^2, "inner" by
    -<x, y> (the largest inner products first)."""

    def __init__(self, comparator):
        self.c = COMPARATORS[comparator]

    def __enter__(self):
        _dir_lock.acquire()
        _load().orc_set_comparator(self.c)

    def __exit__(self, *exc):
        _load().orc_set_comparator(0)
        _dir_lock.release()


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(points), dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("points must be n x m")
    return a


def _graph(idx) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
    if a.ndim != 2:
        raise ValueError("idx must be n x K")
    return a


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def stream_words(seed: int, c0: int, c1: int, c2: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    _load().orc_stream_words(seed, c0, c1, c2, count, _p(out))
    return out


def bounded_draws(seed: int, c0: int, c1: int, c2: int, N: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    _load().orc_bounded_draws(seed, c0, c1, c2, N, count, _p(out))
    return out


def logs(points):
    """(L, negH): L = log(points) elementwise, negH[x] = sum_i x_i log x_i."""
    p = _pts(points)
    n, m = p.shape
    L = np.zeros((n, m))
    negH = np.zeros(n)
    _load().orc_logs(_p(p), n, m, _p(L), _p(negH))
    return L, negH


def keys_pairs(points, xs, ys, comparator: str = "kl") -> np.ndarray:
    """Canonical FP64 key of each pair under the comparator: "kl" negH(x) - <x, log y>,
    "kl_reverse" the same with the roles swapped (D(y||x)), "sqeuclidean"
    (|x|^2 - 2 <x, y>) + |y|^2, "inner" 0 - <x, y>."""
    p = _pts(points)
    n, m = p.shape
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.zeros(len(xs))
    with _comparator(comparator):
        _load().orc_keys_pairs(_p(p), n, m, _p(xs), _p(ys), len(xs), _p(out))
    return out


def init_graph(points, K: int, seed: int, comparator: str = "kl"):
    """Initial random K-out graph (idx n x K int32, key n x K float64), rows sorted."""
    p = _pts(points)
    n, m = p.shape
    idx = np.zeros((n, K), dtype=np.int32)
    key = np.zeros((n, K))
    with _comparator(comparator):
        _load().orc_init_graph(_p(p), n, m, K, seed, _p(idx), _p(key))
    return idx, key


def round_(points, idx_in, x0: int = 0, x1: int | None = None, comparator: str = "kl"):
    """One synchronous round from graph idx_in.  Rows [x0, x1) are computed.

    Returns (idx, key, newflag, updates, proposals); rows outside [x0, x1) of
    the outputs are zero."""
    p = _pts(points)
    g = _graph(idx_in)
    n, m = p.shape
    K = g.shape[1]
    if x1 is None:
        x1 = n
    idx = np.zeros((n, K), dtype=np.int32)
    key = np.zeros((n, K))
    flag = np.zeros((n, K), dtype=np.uint8)
    props = np.zeros(1, dtype=np.int64)
    with _comparator(comparator):
        upd = _load().orc_round(_p(p), n, m, K, _p(g), x0, x1, _p(idx), _p(key), _p(flag), _p(props))
    return idx, key, flag, int(upd), int(props[0])


def indegree(idx) -> np.ndarray:
    g = _graph(idx)
    n, K = g.shape
    deg = np.zeros(n, dtype=np.int64)
    _load().orc_indegree(_p(g), n, K, _p(deg))
    return deg


def pools(idx, x0: int = 0, x1: int | None = None):
    """Candidate pools (sorted sets) of rows [x0, x1) as a list of arrays."""
    g = _graph(idx)
    n, K = g.shape
    if x1 is None:
        x1 = n
    deg = indegree(g)
    cap = int(((K + deg[x0:x1]) * (K + 1)).sum())
    off = np.zeros(x1 - x0 + 1, dtype=np.int64)
    pool = np.zeros(max(cap, 1), dtype=np.int32)
    _load().orc_pools(_p(g), n, K, x0, x1, _p(off), _p(pool))
    return [pool[off[t]:off[t + 1]].copy() for t in range(x1 - x0)]


def fcc(idx, seed: int, round_no: int, S: int) -> int:
    """Friend clustering hit count of graph idx on S samples of round round_no."""
    g = _graph(idx)
    n, K = g.shape
    return int(_load().orc_fcc(_p(g), n, K, seed, round_no, S))


def build(points, K: int, seed: int, S: int = 10000, max_rounds: int = 64, stop_on_zero: bool = True,
          stop_delta: float = 0.0, comparator: str = "kl"):
    """Full build: returns dict(idx, key, rounds, updates[rounds], hits[rounds+1], proposals).
    stop_delta > 0: also stop after a round with fewer than stop_delta*n*K updates."""
    p = _pts(points)
    n, m = p.shape
    idx = np.zeros((n, K), dtype=np.int32)
    key = np.zeros((n, K))
    upd = np.zeros(max_rounds, dtype=np.int64)
    hits = np.zeros(max_rounds + 1, dtype=np.int64)
    props = np.zeros(1, dtype=np.int64)
    with _comparator(comparator):
        r = _load().orc_build(_p(p), n, m, K, seed, S, max_rounds, int(stop_on_zero), float(stop_delta), _p(idx),
                              _p(key), _p(upd), _p(hits), _p(props))
    return {"idx": idx, "key": key, "rounds": int(r), "updates": upd[:r].copy(),
            "hits": hits[:r + 1].copy(), "proposals": int(props[0])}


def bruteforce(points, K: int, queries=None, comparator: str = "kl"):
    """Exact K-NN lists (by (key, idx)) of the query points."""
    p = _pts(points)
    n, m = p.shape
    q = np.arange(n, dtype=np.int32) if queries is None else np.ascontiguousarray(queries, dtype=np.int32)
    idx = np.zeros((len(q), K), dtype=np.int32)
    key = np.zeros((len(q), K))
    with _comparator(comparator):
        _load().orc_bruteforce(_p(p), n, m, K, _p(q), len(q), _p(idx), _p(key))
    return idx, key


def diameter_exact(idx) -> int:
    g = _graph(idx)
    n, K = g.shape
    return int(_load().orc_diameter_exact(_p(g), n, K))


def diameter_bounds(idx, sweeps: int = 8, seed: int = 0):
    g = _graph(idx)
    n, K = g.shape
    lo = np.zeros(1, dtype=np.int32)
    hi = np.zeros(1, dtype=np.int32)
    _load().orc_diameter_bounds(_p(g), n, K, sweeps, seed, _p(lo), _p(hi))
    return int(lo[0]), int(hi[0])


def num_threads() -> int:
    return int(_load().orc_num_threads())
