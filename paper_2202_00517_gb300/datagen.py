"""Seeded synthetic inputs: Dirichlet(1, ..., 1) points on the probability simplex.

This module only makes inputs; it holds none of the descent's arithmetic.  The
CUDA path and the CPU oracle both receive the arrays it returns.

Recipe: point p (0 <= p < n) reads the Philox4x32-10 word stream with key
(seed low 32 bits, seed high 32 bits) and counter (p, 0, 2, block); coordinate i
takes words 2i and 2i+1, forms the 53-bit integer k = ((w[2i] << 32) | w[2i+1])
>> 11 and the uniform u = (k + 1/2) 2^-53 in (0, 1); e_i = -log(u) is Exp(1)
and x_i = e_i / sum_j e_j, computed in float64 and then stored in the requested
dtype.  Normalised independent Exp(1) variables are Dirichlet(1, ..., 1), i.e.
uniform on the simplex, the sampling the paper uses for its experiments
(Sec. 4.4, Sec. 4.5).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def _philox_blocks(c0: np.ndarray, c1: int, c2: int, c3: int, seed: int) -> np.ndarray:
    """Philox4x32-10 of counters (c0[i], c1, c2, c3) -> (len(c0), 4) uint32."""
    x0 = c0.astype(np.uint64)
    x1 = np.full_like(x0, c1)
    x2 = np.full_like(x0, c2)
    x3 = np.full_like(x0, c3)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        n0 = (p1 >> np.uint64(32)) ^ x1 ^ np.uint64(k0)
        n1 = p1 & _MASK
        n2 = (p0 >> np.uint64(32)) ^ x3 ^ np.uint64(k1)
        n3 = p0 & _MASK
        x0, x1, x2, x3 = n0, n1, n2, n3
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return np.stack([x0, x1, x2, x3], axis=1).astype(np.uint32)


def _rows(start: int, stop: int, m: int, seed: int) -> np.ndarray:
    """Points start..stop-1 of the stream, float64, shape (stop - start, m)."""
    nblocks = (2 * m + 3) // 4
    c0 = np.arange(start, stop, dtype=np.uint64)
    words = np.concatenate([_philox_blocks(c0, 0, 2, j, seed) for j in range(nblocks)], axis=1)
    hi = words[:, 0:2 * m:2].astype(np.uint64)
    lo = words[:, 1:2 * m:2].astype(np.uint64)
    k = ((hi << np.uint64(32)) | lo) >> np.uint64(11)
    u = (k.astype(np.float64) + 0.5) * (2.0 ** -53)
    e = -np.log(u)
    return e / e.sum(axis=1, keepdims=True)


def dirichlet_points(n: int, m: int, seed: int, dtype=np.float32, chunk: int = 1 << 18,
                     threads: int = 1) -> np.ndarray:
    """n points uniform on the (m-1)-simplex (m coordinates), shape (n, m).
    The values do not depend on `chunk` or `threads` (host threads over row chunks)."""
    if n < 0 or m < 1:
        raise ValueError("need n >= 0, m >= 1")
    out = np.empty((n, m), dtype=dtype)

    def part(start):
        stop = min(n, start + chunk)
        out[start:stop] = _rows(start, stop, m, seed).astype(dtype)

    starts = range(0, n, chunk)
    if threads > 1:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(part, starts))
    else:
        for st in starts:
            part(st)
    return out


def skewed_points(n: int, m: int, seed: int, power: float, dtype=np.float32) -> np.ndarray:
    """Points near the faces of the simplex: the Dirichlet(1) points of
    `dirichlet_points`, each coordinate raised to `power` in float64 and the row
    renormalised to sum 1, then stored in the requested dtype.  For power > 1 a
    few coordinates carry most of each row's mass and the rest spread over many
    orders of magnitude (down to about 1e-40 at power 8 and m = 11)."""
    x = dirichlet_points(n, m, seed, np.float64) ** power
    return (x / x.sum(axis=1, keepdims=True)).astype(dtype)


def instance_mix(count: int, seed: int):
    """Shapes of a batch of independent instances: n log-uniform in [200, 50000],
    m in {6, 11, 21}, K in {8, 16, 32}, each uniform, drawn from the Philox stream
    (seed, counter (i, 0, 4, block)) of instance i.  Returns a list of
    (n, m, K) tuples."""
    c0 = np.arange(count, dtype=np.uint64)
    w = _philox_blocks(c0, 0, 4, 0, seed)
    u = (w[:, 0].astype(np.float64) + 0.5) * 2.0 ** -32
    n = np.floor(200.0 * 250.0 ** u).astype(np.int64)
    n = np.clip(n, 200, 50000)
    ms = np.array([6, 11, 21])[w[:, 1] % 3]
    ks = np.array([8, 16, 32])[w[:, 2] % 3]
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, ms, ks)]
