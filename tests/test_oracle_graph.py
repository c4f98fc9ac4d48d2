"""Pins of the oracle's graph steps: initial random K-out graph (Sec. 3.2),
one synchronous round (Sec. 3.1, Sec. 4.2), brute-force K-NN (Sec. 2.3), the
friend clustering rate (Sec. 3.3) and the BFS diameter (Sec. 3.2, Sec. 4.3).

The round is checked against an independent pure-Python enumeration of the
pools (Python sets, keys from scipy's relative entropy), against the exact
K-NN graph where the method must reach it, and against invariants that hold
for every synchronous round."""
import networkx as nx
import numpy as np
import pytest
from scipy import stats
from scipy.spatial.distance import cdist
from scipy.special import rel_entr

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points


def _scipy_keys(p, x, ys, comparator="kl"):
    if comparator == "kl_reverse":  # y ranked for x by D(y||x)
        return rel_entr(p[ys], p[x][None, :]).sum(1)
    if comparator == "sqeuclidean":
        return cdist(p[x][None, :], p[ys], "sqeuclidean")[0]
    if comparator == "inner":
        return -(p[ys] @ p[x])
    return rel_entr(p[x][None, :], p[ys]).sum(1)


def _check_rows(idx, key, n, K):
    assert idx.shape == (n, K)
    assert np.all(idx >= 0) and np.all(idx < n)
    assert np.all(idx != np.arange(n)[:, None]), "self as friend"
    s = np.sort(idx, axis=1)
    assert np.all(s[:, 1:] != s[:, :-1]), "duplicate friend"
    # sorted by (key, idx)
    d = np.diff(key, axis=1)
    assert np.all((d > 0) | ((d == 0) & (idx[:, 1:] > idx[:, :-1])))


# ---------------------------------------------------------------- initial graph
def test_init_graph_shape_and_order():
    n, m, K = 2000, 6, 10
    p = dirichlet_points(n, m, 0, np.float64)
    idx, key = oracle.init_graph(p, K, 0)
    _check_rows(idx, key, n, K)
    rows = np.repeat(np.arange(n), K)
    assert np.array_equal(key.ravel(), oracle.keys_pairs(p, rows, idx.ravel()))
    # deterministic in the seed, different across seeds
    idx2, _ = oracle.init_graph(p, K, 0)
    assert np.array_equal(idx, idx2)
    idx3, _ = oracle.init_graph(p, K, 1)
    assert not np.array_equal(idx, idx3)


def test_init_graph_uniform():
    n, m, K = 2000, 6, 10
    p = dirichlet_points(n, m, 0, np.float64)
    idx, _ = oracle.init_graph(p, K, 0)
    # offsets (y - x) mod n are uniform on 1..n-1
    off = (idx - np.arange(n)[:, None]) % n
    counts = np.bincount(((off.ravel() - 1) * 20) // (n - 1), minlength=20)
    assert stats.chisquare(counts).pvalue > 1e-4
    # in-degree ~ Binomial(n-1, K/(n-1)): mean K exactly, variance close to K
    deg = oracle.indegree(idx)
    assert deg.sum() == n * K
    assert 0.8 * K < deg.var() < 1.2 * K


# ---------------------------------------------------------------- one round
def _python_pool(idx, x):
    n, K = idx.shape
    F = [set(map(int, r)) for r in idx]
    coF = [set() for _ in range(n)]
    for a in range(n):
        for b in idx[a]:
            coF[int(b)].add(a)
    pool = set(F[x]) | coF[x]
    for v in F[x]:
        pool |= F[v]
    for w in coF[x]:
        pool |= F[w]
    pool.discard(x)
    return pool


@pytest.mark.parametrize("comparator", ["kl", "kl_reverse", "sqeuclidean", "inner"])
def test_round_equals_independent_pool_topk(comparator):
    n, m, K = 80, 4, 5
    p = dirichlet_points(n, m, 21, np.float64)
    if comparator in ("sqeuclidean", "inner"):  # any finite coordinates
        p = np.random.default_rng(21).standard_normal((n, m))
    idx0, _ = oracle.init_graph(p, K, 21, comparator=comparator)
    pools = oracle.pools(idx0)
    idx1, key1, flag, upd, props = oracle.round_(p, idx0, comparator=comparator)
    _check_rows(idx1, key1, n, K)
    newcount = 0
    for x in range(n):
        pool = sorted(_python_pool(idx0, x))
        assert np.array_equal(pools[x], np.array(pool)), x
        keys = _scipy_keys(p, x, np.array(pool), comparator)
        order = np.lexsort((np.array(pool), keys))
        best = np.array(pool)[order[:K]]
        kb = keys[order[:K + 1]]
        # a reordering is allowed only where two keys are within rounding of each other
        if np.all(np.diff(kb) > 1e-12):
            assert np.array_equal(idx1[x], best), x
        else:
            assert set(idx1[x]) <= set(pool)
        assert np.allclose(key1[x], keys[order[:K]], rtol=0, atol=1e-13)
        old = set(map(int, idx0[x]))
        fl = np.array([0 if int(y) in old else 1 for y in idx1[x]], dtype=np.uint8)
        assert np.array_equal(flag[x], fl)
        newcount += int(fl.sum())
    assert upd == newcount
    assert props == n * (K + 2 * K * K)


def test_round_complete_graph_is_fixed_point():
    # n = K+1: the initial graph already holds every other point, so it is the
    # exact K-NN graph and a round changes nothing.
    K = 7
    n = K + 1
    p = dirichlet_points(n, 5, 4, np.float64)
    idx0, key0 = oracle.init_graph(p, K, 4)
    bi, bk = oracle.bruteforce(p, K)
    assert np.array_equal(idx0, bi) and np.array_equal(key0, bk)
    idx1, key1, flag, upd, _ = oracle.round_(p, idx0)
    assert upd == 0 and np.all(flag == 0)
    assert np.array_equal(idx1, idx0) and np.array_equal(key1, key0)


def test_round_invariants_over_build():
    n, m, K = 1500, 6, 8
    p = dirichlet_points(n, m, 3, np.float64)
    idx, key = oracle.init_graph(p, K, 3)
    for r in range(1, 7):
        nidx, nkey, flag, upd, _ = oracle.round_(p, idx)
        _check_rows(nidx, nkey, n, K)
        # old friends stay in the pool: sorted keys never get worse
        assert np.all(nkey <= key)
        assert upd == int(flag.sum())
        if upd == 0:
            assert np.array_equal(nidx, idx)
        idx, key = nidx, nkey
    # a second round from a fixed point is a fixed point
    nidx, nkey, _, upd, _ = oracle.round_(p, idx)
    if upd == 0:
        assert np.array_equal(nidx, idx)


def test_round_row_range():
    n, m, K = 500, 5, 6
    p = dirichlet_points(n, m, 8, np.float64)
    idx0, _ = oracle.init_graph(p, K, 8)
    full = oracle.round_(p, idx0)
    part = oracle.round_(p, idx0, 100, 250)
    assert np.array_equal(full[0][100:250], part[0][100:250])
    assert np.array_equal(full[1][100:250], part[1][100:250])
    assert part[3] == int(full[2][100:250].sum())


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("comparator", ["kl", "kl_reverse", "sqeuclidean", "inner"])
def test_bruteforce_matches_full_matrix(comparator):
    n, m, K = 300, 6, 9
    p = dirichlet_points(n, m, 13, np.float64)
    bi, bk = oracle.bruteforce(p, K, comparator=comparator)
    D = rel_entr(p[:, None, :], p[None, :, :]).sum(-1)  # D[x, y] = D(x||y)
    if comparator == "kl_reverse":
        D = D.T.copy()  # row x: D(y||x)
    elif comparator == "sqeuclidean":
        D = cdist(p, p, "sqeuclidean")
    elif comparator == "inner":
        D = -(p @ p.T)
    np.fill_diagonal(D, np.inf)
    for x in range(n):
        order = np.lexsort((np.arange(n), D[x]))[:K]
        assert np.array_equal(bi[x], order), x
        assert np.allclose(bk[x], D[x][order], atol=1e-13, rtol=0)


# ---------------------------------------------------------------- clustering rate
def _cayley(n, A):
    A = np.array(A)
    return ((np.arange(n)[:, None] + A[None, :]) % n).astype(np.int32)


def test_ties_ordered_by_index():
    # Exact copies of a point key to exactly 0 against it (the same chain on the
    # same numbers), so equal keys meet; the order is (key, index) ascending.
    n, K = 300, 8
    p = dirichlet_points(n, 6, 8, np.float64)
    dups = [17, 45, 101, 150, 299]
    p[dups] = p[3]
    bi, bk = oracle.bruteforce(p, K, [3])
    assert list(bi[0, :5]) == dups and np.all(bk[0, :5] == 0.0)
    assert np.all(bk[0, 5:] > 0.0)
    # a copy sees the original and the other copies, lowest index first
    bi, bk = oracle.bruteforce(p, K, [150])
    assert list(bi[0, :5]) == [3, 17, 45, 101, 299] and np.all(bk[0, :5] == 0.0)
    # a round on many copies meets ties and still orders them by index
    q = dirichlet_points(n, 6, 9, np.float64)
    q[1::3] = q[0::3][: len(q[1::3])]
    g0, _ = oracle.init_graph(q, K, 9)
    idx, key, _, _, _ = oracle.round_(q, g0)
    _check_rows(idx, key, n, K)
    assert np.any(np.diff(key, axis=1) == 0)


def test_fcc_complete_graph_always_hits():
    K = 6
    idx = np.array([[y for y in range(K + 1) if y != x] for x in range(K + 1)], dtype=np.int32)
    assert oracle.fcc(idx, 1, 3, 5000) == 5000


def test_fcc_odd_generators_never_hit():
    # F(x) = x + {1, 3, ..., 2K-1} mod n with n even: differences of two friends
    # are even, so no friend is a friend or co-friend of another.
    n, K = 1000, 8
    idx = _cayley(n, list(range(1, 2 * K, 2)))
    assert oracle.fcc(idx, 2, 1, 5000) == 0


def test_fcc_consecutive_generators_always_hit():
    n, K = 1000, 8
    idx = _cayley(n, list(range(1, K + 1)))
    assert oracle.fcc(idx, 3, 2, 5000) == 5000


def test_fcc_partial_rate():
    # A = {1, 2, 4}: of the 3 unordered friend pairs, {1,2} and {2,4} hit
    # (differences 1 and 2 are generators), {1,4} does not (3 is not).
    n, S = 997, 30000
    idx = _cayley(n, [1, 2, 4])
    h = oracle.fcc(idx, 4, 1, S)
    sd = np.sqrt(S * (2 / 3) * (1 / 3))
    assert abs(h - S * 2 / 3) < 5 * sd


def test_fcc_random_graph_rate():
    n, K, S = 2000, 10, 20000
    p = dirichlet_points(n, 6, 0, np.float64)
    idx, _ = oracle.init_graph(p, K, 0)
    h = oracle.fcc(idx, 0, 0, S)
    rate = 2 * K / (n - 1)
    assert abs(h - S * rate) < 5 * np.sqrt(S * rate)


def test_fcc_rounds_draw_fresh_samples():
    # The clustering rate is estimated afresh in every round (Sec. 3.3): on one
    # fixed graph with exact hit rate 2/3 (generators {1, 2, 4}), the counts of
    # forty rounds scatter like independent binomial draws, not like one draw
    # repeated.
    n, S, R = 997, 2000, 40
    idx = _cayley(n, [1, 2, 4])
    h = np.array([oracle.fcc(idx, 6, r, S) for r in range(R)], dtype=np.float64)
    p = 2 / 3
    assert abs(h.mean() - S * p) < 5 * np.sqrt(S * p * (1 - p) / R)
    ratio = h.var(ddof=1) / (S * p * (1 - p))
    lo, hi = stats.chi2.ppf([1e-6, 1 - 1e-6], R - 1) / (R - 1)
    assert lo < ratio < hi
    # the seed enters every sample as well
    assert [oracle.fcc(idx, 7, r, S) for r in range(4)] != list(h[:4].astype(int))


def test_fcc_draws_x_over_all_points():
    # Sec. 3.3 samples x uniformly from all n points.  Points 0..499 sit in cliques
    # of five (any two friends are friends: always a hit); points 500..999 form a
    # ring with odd offsets {1, 3, 5, 7} (two friends differ by an even step, never
    # a friend: never a hit).  The hit rate is exactly 1/2.
    n, K, S = 1000, 4, 20000
    idx = np.zeros((n, K), dtype=np.int32)
    for x in range(500):
        b = x - x % 5
        idx[x] = [y for y in range(b, b + 5) if y != x]
    for x in range(500, 1000):
        idx[x] = [500 + (x - 500 + a) % 500 for a in (1, 3, 5, 7)]
    h = oracle.fcc(idx, 5, 1, S)
    assert abs(h - S / 2) < 5 * np.sqrt(S / 4)


# ---------------------------------------------------------------- diameter
@pytest.mark.parametrize("n,K,seed", [(200, 3, 1), (500, 4, 2), (1200, 3, 3)])
def test_diameter_matches_networkx(n, K, seed):
    p = dirichlet_points(n, 4, seed, np.float64)
    idx, _ = oracle.init_graph(p, K, seed)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((x, int(y)) for x in range(n) for y in idx[x])
    d = nx.diameter(G)
    assert oracle.diameter_exact(idx) == d
    lo, hi = oracle.diameter_bounds(idx, sweeps=6, seed=seed)
    assert lo <= d <= hi


def test_diameter_path_graph():
    # K = 1 ring 0 -> 1 -> ... -> n-1 -> 0: undirected cycle, diameter n // 2
    n = 101
    idx = ((np.arange(n) + 1) % n).astype(np.int32)[:, None]
    assert oracle.diameter_exact(idx) == n // 2


def test_diameter_disconnected_graph():
    # two disjoint 3-out rings: no path between them, so no finite diameter
    n, K = 400, 3
    idx = np.zeros((n, K), dtype=np.int32)
    for x in range(n):
        b = 0 if x < 200 else 200
        idx[x] = [b + (x - b + a) % 200 for a in (1, 2, 3)]
    assert oracle.diameter_exact(idx) == -1
    assert oracle.diameter_bounds(idx, 4, 1) == (-1, -1)
    # joined by one arc the graph is connected again
    idx[0, 0] = 200
    assert oracle.diameter_exact(idx) > 0


def test_diameter_bounds_use_every_sweep():
    # Every double sweep raises the lower bound to the largest eccentricity seen:
    # on sparse random graphs one sweep finds the exact diameter less than half
    # the time, twenty sweeps nearly always; every bracket holds.
    hits = 0
    for seed in range(40):
        p = dirichlet_points(300, 3, seed, np.float64)
        g, _ = oracle.init_graph(p, 2, seed)
        ex = oracle.diameter_exact(g)
        lo1, hi1 = oracle.diameter_bounds(g, 1, seed)
        lo, hi = oracle.diameter_bounds(g, 20, seed)
        assert lo1 <= lo <= ex <= hi <= hi1
        hits += lo == ex
    assert hits >= 32
