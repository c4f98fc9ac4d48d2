"""Pins of the oracle's KL comparator key (Sec. 2.2): key(x, y) = D(x||y).

Each check ties the oracle to something outside itself: hand-worked closed forms,
scipy's elementwise relative entropy, the closed form for a uniform y, and the
exact zero of D(x||x).  A transposed operand (D(y||x)), a dropped -H(x) term or
a sign error fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy.special import rel_entr

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kl_worked_example.txt")


def _read_golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        xs, ys, _form, val = [s.strip() for s in line.split(";")]
        rows.append((np.array([float(t) for t in xs.split(",")]),
                     np.array([float(t) for t in ys.split(",")]), float(val)))
    return rows


def test_worked_examples():
    for x, y, val in _read_golden():
        k = oracle.keys_pairs(np.stack([x, y]), [0], [1])[0]
        assert abs(k - val) <= 4e-16 * max(1.0, abs(val)) * 8, (x, y, k, val)


def test_direction_is_x_first():
    # D(x||y) != D(y||x) in the worked examples: the key must weight by x.
    x, y, val = _read_golden()[0]
    k_xy = oracle.keys_pairs(np.stack([x, y]), [0], [1])[0]
    k_yx = oracle.keys_pairs(np.stack([x, y]), [1], [0])[0]
    assert abs(k_xy - val) < 1e-15
    assert abs(k_yx - val) > 1e-3


def test_self_key_is_exactly_zero():
    p = dirichlet_points(300, 7, 11, np.float64)
    xs = np.arange(300)
    k = oracle.keys_pairs(p, xs, xs)
    assert np.all(k == 0.0)


def test_matches_scipy_relative_entropy():
    p = dirichlet_points(400, 21, 5, np.float64)
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 400, 5000)
    ys = rng.integers(0, 400, 5000)
    k = oracle.keys_pairs(p, xs, ys)
    ref = rel_entr(p[xs], p[ys]).sum(axis=1)
    # scale of the terms: |negH(x)| + sum_i x_i |log y_i|
    scale = np.abs((p[xs] * np.log(p[xs])).sum(1)) + (p[xs] * np.abs(np.log(p[ys]))).sum(1)
    assert np.all(np.abs(k - ref) <= 1e-13 * scale)


def test_uniform_y_closed_form():
    # y uniform: D(x||u) = sum_i x_i log x_i + log(m) sum_i x_i
    m = 9
    p = dirichlet_points(50, m, 3, np.float64)
    u = np.full((1, m), 1.0 / m)
    pts = np.concatenate([p, u])
    k = oracle.keys_pairs(pts, np.arange(50), np.full(50, 50))
    ref = (p * np.log(p)).sum(1) + np.log(m) * p.sum(1)
    assert np.allclose(k, ref, rtol=0, atol=1e-14)


def test_gibbs_nonnegative():
    p = dirichlet_points(200, 5, 2, np.float64)
    rng = np.random.default_rng(1)
    xs = rng.integers(0, 200, 3000)
    ys = rng.integers(0, 200, 3000)
    k = oracle.keys_pairs(p, xs, ys)
    assert np.all(k >= -1e-14)


def test_logs_table():
    p = dirichlet_points(100, 6, 9, np.float64)
    L, negH = oracle.logs(p)
    assert np.array_equal(L, np.log(p))
    assert np.allclose(negH, (p * np.log(p)).sum(1), rtol=1e-14, atol=0)


def test_reverse_direction_matches_scipy():
    # the variant comparator ranks y for x by D(y||x) (scipy: rel_entr(y, x))
    p = dirichlet_points(300, 11, 6, np.float64)
    rng = np.random.default_rng(1)
    xs = rng.integers(0, 300, 3000)
    ys = rng.integers(0, 300, 3000)
    k = oracle.keys_pairs(p, xs, ys, comparator="kl_reverse")
    ref = rel_entr(p[ys], p[xs]).sum(axis=1)
    scale = np.abs((p[ys] * np.log(p[ys])).sum(1)) + (p[ys] * np.abs(np.log(p[xs]))).sum(1)
    assert np.all(np.abs(k - ref) <= 1e-13 * scale)
    # the two directions differ (the divergence is not symmetric) but agree on x = y
    assert np.max(np.abs(k - oracle.keys_pairs(p, xs, ys))) > 1e-3
    same = oracle.keys_pairs(p, np.arange(300), np.arange(300), comparator="kl_reverse")
    assert np.all(same == oracle.keys_pairs(p, np.arange(300), np.arange(300)))


def test_squared_euclidean_matches_numpy():
    # the metric comparator: (|x|^2 - 2<x, y>) + |y|^2, for any finite coordinates
    p = np.random.default_rng(2).standard_normal((300, 13)) * 3.0
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 300, 3000)
    ys = rng.integers(0, 300, 3000)
    k = oracle.keys_pairs(p, xs, ys, comparator="sqeuclidean")
    ref = ((p[xs] - p[ys]) ** 2).sum(1)
    scale = (p[xs] ** 2).sum(1) + (p[ys] ** 2).sum(1)
    assert np.all(np.abs(k - ref) <= 1e-14 * scale)
    # symmetric, up to the last rounding of the two orders of the sum
    assert np.allclose(k, oracle.keys_pairs(p, ys, xs, comparator="sqeuclidean"), rtol=0, atol=1e-14 * scale.max())


def test_inner_product_matches_numpy():
    # maximum inner product neighbours: key 0 - <x, y>, any finite coordinates
    p = np.random.default_rng(5).standard_normal((300, 13)) * 2.0
    rng = np.random.default_rng(6)
    xs = rng.integers(0, 300, 3000)
    ys = rng.integers(0, 300, 3000)
    k = oracle.keys_pairs(p, xs, ys, comparator="inner")
    ref = -(p[xs] * p[ys]).sum(1)
    scale = (np.abs(p[xs]) * np.abs(p[ys])).sum(1)
    assert np.all(np.abs(k - ref) <= 1e-14 * scale)
    # the chain is the KL form's with L = x and negH = 0: exact sign of an empty sum
    z = np.zeros((2, 3))
    kz = oracle.keys_pairs(z, [0], [1], comparator="inner")[0]
    assert kz == 0.0 and not np.signbit(kz)  # 0 - (+0) = +0
    # not a metric: a point need not be its own best match
    q = np.array([[1.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    kk = oracle.keys_pairs(q, [0, 0], [1, 0], comparator="inner")
    assert kk[0] < kk[1]
