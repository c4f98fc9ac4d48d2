"""The synthetic input generator: points lie in the open simplex, are
reproducible from the seed, and follow Dirichlet(1, ..., 1) (each coordinate's
marginal is Beta(1, m-1), with CDF 1 - (1 - t)^(m-1))."""
import numpy as np
from scipy import stats

from paper_2202_00517_gb300.datagen import dirichlet_points, instance_mix, skewed_points


def test_points_on_simplex_and_reproducible():
    p = dirichlet_points(5000, 21, 1, np.float64)
    assert p.shape == (5000, 21)
    assert np.all(p > 0) and np.all(p < 1)
    assert np.allclose(p.sum(1), 1.0, atol=1e-14)
    assert np.array_equal(p, dirichlet_points(5000, 21, 1, np.float64))
    assert not np.array_equal(p, dirichlet_points(5000, 21, 2, np.float64))
    p32 = dirichlet_points(5000, 21, 1, np.float32)
    assert p32.dtype == np.float32 and np.array_equal(p32, p.astype(np.float32))
    # chunking does not change the values
    assert np.array_equal(p, dirichlet_points(5000, 21, 1, np.float64, chunk=777))


def test_dirichlet_marginals():
    m = 6
    p = dirichlet_points(20000, m, 4, np.float64)
    for i in (0, 3, 5):
        assert stats.kstest(p[:, i], lambda t: 1 - (1 - t) ** (m - 1)).pvalue > 1e-4


def test_instance_mix():
    mix = instance_mix(4096, 5)
    ns = np.array([a for a, _, _ in mix])
    assert ns.min() >= 200 and ns.max() <= 50000
    assert {b for _, b, _ in mix} == {6, 11, 21}
    assert {c for _, _, c in mix} == {8, 16, 32}
    # log-uniform: log(n/200)/log(250) is close to uniform
    u = np.log(ns / 200) / np.log(250)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert mix == instance_mix(4096, 5)


def test_threads_and_chunks_do_not_change_values():
    a = dirichlet_points(3000, 7, 9, np.float32)
    b = dirichlet_points(3000, 7, 9, np.float32, chunk=256, threads=4)
    assert np.array_equal(a, b)


def test_skewed_points():
    p = skewed_points(500, 11, 3, 16, np.float64)
    assert p.shape == (500, 11) and np.all(p > 0)
    assert np.allclose(p.sum(1), 1.0, rtol=0, atol=1e-15)
    # most of each row's mass on few coordinates, the rest over many decades
    assert np.median(p.max(1)) > 0.5 and p.min() < 1e-40
    q = dirichlet_points(500, 11, 3, np.float64) ** 16
    assert np.array_equal(p, q / q.sum(1, keepdims=True))
