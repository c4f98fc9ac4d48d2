"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

* initial graph: identical index lists, keys within the tie tolerance;
* lockstep rounds: every CUDA round is fed the oracle's previous graph and must
  return the oracle's next graph (index lists identical except near-ties),
  the same update count and the same clustering hits;
* free-running builds: identical rounds, updates, hits and graphs;
* the mixed form equals the FP64 form bit for bit;
* incremental proposals (a pair met only through arcs of the previous round's
  graph is not proposed again) give the same graph as proposing every pair;
  lockstep rounds run both ways against the oracle's full pool;
* shapes spanning several warps/tiles with ragged tails, K from 2 to 64, m from
  1 (every key ties) to 128, n = K+1, duplicated points (exact ties), points near
  the simplex's faces (coordinates that underflow in the FP32 filter).
"""
import numpy as np
import pytest

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points, skewed_points
from parity_util import check_invariants, compare_graphs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# "mixed_tma": the mixed form with the TMA-gathered join forced (by default it runs
# from n = 65,536 on; these shapes are smaller)
PRECS = ("fp64", "mixed", "mixed_tma", "bf16x3")


def _handle(knnd, *args, precision="mixed", **kw):
    if precision == "mixed_tma":
        precision, kw["join_form"] = "mixed", "tma"
    return knnd.Handle(*args, precision=precision, **kw)


@pytest.fixture(scope="module")
def knnd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2202_00517_gb300 as k
    return k


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _lockstep(knnd, pts, K, seed, prec, rounds, dtype="f64", S=2000, incremental=True, comparator="kl"):
    n, m = pts.shape
    p = _dev(pts)
    h = _handle(knnd, n, m, K, dtype=dtype, precision=prec, fcc_samples=S, incremental=incremental,
                    comparator=comparator)
    pts64 = pts.astype(np.float64)
    gi, gk, _ = h.init_graph(p, seed)
    ri, rk = oracle.init_graph(pts64, K, seed, comparator=comparator)
    assert np.array_equal(gi.cpu().numpy(), ri)
    compare_graphs(pts64, gi.cpu().numpy(), gk.cpu().numpy(), ri, rk, max_tie_rows=0, comparator=comparator)
    upd = torch.zeros(1, dtype=torch.int64, device="cuda")
    hits = torch.zeros(1, dtype=torch.int64, device="cuda")
    total_ties = 0
    rf = np.ones(ri.shape, dtype=np.uint8)  # new-flags of the oracle's graph (read when incremental)
    for r in range(1, rounds + 1):
        idx = _dev(ri)
        key = _dev(rk)
        flag = _dev(rf)
        h.round(None, seed, r, idx, key, flag, upd, hits)
        h.sync()
        ni, nk, nf, nu, _ = oracle.round_(pts64, ri, comparator=comparator)
        ties = compare_graphs(pts64, idx.cpu().numpy(), key.cpu().numpy(), ni, nk, comparator=comparator)
        total_ties += ties
        if ties == 0:
            assert np.array_equal(idx.cpu().numpy(), ni)
            assert np.array_equal(flag.cpu().numpy(), nf)
            assert int(upd.item()) == nu
            assert int(hits.item()) == oracle.fcc(ni, seed, r, S)
        check_invariants(idx.cpu().numpy(), key.cpu().numpy())
        ri, rk, rf = ni, nk, nf
    h.close()
    return total_ties


@pytest.mark.parametrize("prec", PRECS)
def test_config1_lockstep(knnd, prec):
    pts = dirichlet_points(2000, 6, 0, np.float64)
    assert _lockstep(knnd, pts, 10, 0, prec, rounds=6) == 0


@pytest.mark.parametrize("prec", PRECS)
def test_config1_build_equals_oracle(knnd, prec):
    n, m, K, seed = 2000, 6, 10, 0
    pts = dirichlet_points(n, m, seed, np.float64)
    ref = oracle.build(pts, K, seed)
    h = _handle(knnd, n, m, K, dtype="f64", precision=prec)
    out = h.build(_dev(pts), seed)
    assert out["rounds"] == ref["rounds"]
    assert out["updates"] == list(ref["updates"])
    assert out["fcc_hits"] == list(ref["hits"])
    assert out["proposals"] == ref["rounds"] * n * (K + 2 * K * K) == ref["proposals"]
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
    compare_graphs(pts, out["idx"].cpu().numpy(), out["key"].cpu().numpy(), ref["idx"], ref["key"], max_tie_rows=0)
    # host-memory entry point returns the same graph
    hb = h.build_host(torch.from_numpy(pts).pin_memory(), seed)
    assert np.array_equal(hb["idx"].numpy(), ref["idx"])
    assert np.array_equal(hb["key"].numpy(), out["key"].cpu().numpy())
    h.close()


SHAPES = [
    # n, m, K, seed, dtype
    (3, 2, 2, 1, "f64"),
    (50, 1, 4, 2, "f64"),        # m = 1: every point is (1), every key is 0; order by index
    (33, 3, 32, 3, "f64"),       # n = K + 1: complete graph, fixed point
    (100, 2, 2, 4, "f32"),
    (777, 11, 16, 5, "f32"),
    (1001, 21, 33, 6, "f32"),    # K > 32: two list slots per lane, two columns per lane
    (1500, 65, 32, 7, "f32"),
    (600, 128, 64, 8, "f64"),
    (2500, 24, 20, 9, "f32"),
    (1200, 40, 17, 10, "f32"),   # 40 coordinates (48 padded), odd K
    (1300, 19, 20, 11, "f32"),   # 19 coordinates (24 padded)
    (900, 10, 40, 12, "f64"),    # 10 coordinates (16 padded) with K > 32
]


@pytest.mark.parametrize("n,m,K,seed,dtype", SHAPES)
@pytest.mark.parametrize("prec", PRECS)
def test_shapes_lockstep(knnd, n, m, K, seed, dtype, prec):
    pts = dirichlet_points(n, m, seed, np.float32 if dtype == "f32" else np.float64)
    ties = _lockstep(knnd, pts, K, seed, prec, rounds=3, dtype=dtype, S=500)
    assert ties <= max(2, n // 500)


@pytest.mark.parametrize("dtype,power", [("f64", 16), ("f32", 4)])
@pytest.mark.parametrize("prec", PRECS)
def test_skewed_points_lockstep(knnd, prec, dtype, power):
    # Points near the faces of the simplex.  In FP64 (power 16) coordinates go down
    # to about 1e-73: the filter's FP32 copy turns some into subnormals and some
    # into 0, and |log y| reaches about 170, so the FP32 bound is wide and most
    # pairs reach the FP64 re-score.  The graphs must still be the oracle's, with
    # no audited bound violation, and every form must equal the FP64 form.
    n, m, K, seed = 1500, 11, 16, 31
    pts = skewed_points(n, m, seed, power, np.float64 if dtype == "f64" else np.float32)
    assert np.all(pts > 0)
    if dtype == "f64":
        assert np.any(pts.astype(np.float32) == 0)  # the case this test is for
    ties = _lockstep(knnd, pts, K, seed, prec, rounds=3, dtype=dtype, S=500)
    assert ties <= max(2, n // 500)
    p = _dev(pts)
    h = _handle(knnd, n, m, K, dtype=dtype, precision=prec, debug=True)
    out = h.build(p, seed)
    h.close()
    assert out["bound_violations"] == 0
    ref = _handle(knnd, n, m, K, dtype=dtype, precision="fp64")
    r = ref.build(p, seed)
    ref.close()
    assert torch.equal(out["idx"], r["idx"]) and torch.equal(out["key"], r["key"])


@pytest.mark.parametrize("prec", PRECS)
def test_duplicated_points_exact_ties(knnd, prec):
    base = dirichlet_points(300, 5, 11, np.float64)
    pts = np.repeat(base, 3, axis=0)  # every point three times: exact key ties
    # Lockstep feeds the oracle's stored keys (C-library log) next to keys the
    # CUDA path computes (CUDA log): two copies of one point may then differ in
    # the last bit, a near-tie the comparison accepts and counts.
    assert _lockstep(knnd, pts, 8, 11, prec, rounds=3, S=500) <= len(pts) // 100
    # Free-running, each side keys every copy identically: ties go by index and
    # the graphs must be identical.
    ref = oracle.build(pts, 8, 11, S=500)
    h = _handle(knnd, len(pts), 5, 8, dtype="f64", precision=prec, fcc_samples=500)
    out = h.build(_dev(pts), 11)
    h.close()
    assert out["rounds"] == ref["rounds"] and out["updates"] == list(ref["updates"])
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])


@pytest.mark.parametrize("prec", PRECS)
def test_lockstep_all_pairs_proposed(knnd, prec):
    # incremental proposals off: every pair the tiles meet goes to the merge
    pts = dirichlet_points(3000, 11, 12, np.float32)
    assert _lockstep(knnd, pts, 12, 12, prec, rounds=4, dtype="f32", S=500, incremental=False) <= 6


@pytest.mark.parametrize("n,m,K", [(100_000, 21, 20), (30_000, 65, 32), (20_000, 6, 8)])
def test_incremental_proposals_same_graph(knnd, n, m, K):
    # a pair met only through arcs of the previous round's graph is not proposed
    # again: the build is the same, bit for bit, with fewer candidates merged
    # The TMA join takes no incremental proposals, so in the mixed form both builds
    # join with plain loads (the survivor counts then compare like with like), and
    # the full pool joined by TMA must give the same graph as well.
    seed = 4
    pts = _dev(dirichlet_points(n, m, seed, np.float32))
    for prec in ("fp64", "mixed", "bf16x3"):
        res = {}
        for inc in (False, True):
            kw = {"join_form": "plain"} if prec == "mixed" else {}
            h = _handle(knnd, n, m, K, dtype="f32", precision=prec, incremental=inc, **kw)
            res[inc] = h.build(pts, seed)
            h.close()
        a, b = res[False], res[True]
        assert a["rounds"] == b["rounds"] and a["updates"] == b["updates"] and a["fcc_hits"] == b["fcc_hits"], prec
        assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["key"], b["key"]), prec
        assert b["join_survivors"] < a["join_survivors"], prec
        if prec == "mixed":
            h = _handle(knnd, n, m, K, dtype="f32", precision="mixed_tma")
            c = h.build(pts, seed)
            h.close()
            assert c["join_kernel"] == "tma", prec
            assert c["updates"] == b["updates"], prec
            assert torch.equal(c["idx"], b["idx"]) and torch.equal(c["key"], b["key"]), prec


@pytest.mark.parametrize("n,m,K", [(200_000, 21, 20), (60_000, 65, 32), (50_000, 11, 32)])
def test_mixed_forms_equal_fp64_bitwise(knnd, n, m, K):
    seed = 1
    pts = _dev(dirichlet_points(n, m, seed, np.float32))
    res = {}
    for prec in PRECS:
        h = _handle(knnd, n, m, K, dtype="f32", precision=prec)
        res[prec] = h.build(pts, seed)
        h.close()
    a = res["fp64"]
    for prec in ("mixed", "mixed_tma", "bf16x3"):
        b = res[prec]
        assert a["rounds"] == b["rounds"] and a["updates"] == b["updates"] and a["fcc_hits"] == b["fcc_hits"], prec
        assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["key"], b["key"]), prec
        assert b["rescored"] > 0
    check_invariants(a["idx"].cpu().numpy(), a["key"].cpu().numpy())


@pytest.mark.parametrize("prec", ["mixed", "mixed_tma", "bf16x3"])
@pytest.mark.parametrize("m,K", [(21, 20), (65, 32), (6, 10)])
def test_error_bound_audit(knnd, prec, m, K):
    # debug mode checks every low-precision dot the tensor-core join and the
    # TMA-gathered FP32 join (up to 32 padded coordinates and K <= 32) compute
    # against the FP64 dot: none may exceed the bound the filter relies on
    n = 6000
    pts = _dev(dirichlet_points(n, m, 17, np.float32))
    h = _handle(knnd, n, m, K, dtype="f32", precision=prec, debug=True)
    out = h.build(pts, 17)
    h.close()
    assert out["bound_violations"] == 0
    if prec == "bf16x3" or (prec == "mixed_tma" and m <= 32 and K <= 32):
        assert out["bound_audited"] > n * K
        assert out["join_kernel"] == ("tc" if prec == "bf16x3" else "tma")
    ref = _handle(knnd, n, m, K, dtype="f32", precision="fp64")
    r = ref.build(pts, 17)
    ref.close()
    assert torch.equal(out["idx"], r["idx"]) and torch.equal(out["key"], r["key"])


def test_domain_errors_and_recovery(knnd):
    n, m, K = 500, 6, 8
    pts = dirichlet_points(n, m, 3, np.float64)
    h = _handle(knnd, n, m, K, dtype="f64", precision="mixed")
    for bad in (0.0, -0.5, np.nan, np.inf):
        q = pts.copy()
        q[123, 4] = bad
        with pytest.raises(knnd.api._lib.KnndError) as e:
            h.build(_dev(q), 3)
        assert e.value.status == knnd.api._lib.KNND_EDOMAIN
    out = h.build(_dev(pts), 3)  # the handle stays usable
    ref = oracle.build(pts, K, 3)
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
    h.close()


def test_out_of_range_indices_are_reported(knnd):
    # The kernels check every graph index they follow; a bad one is skipped and
    # recorded, and knnd_sync reports EINVAL.
    n, m, K = 400, 4, 6
    pts = dirichlet_points(n, m, 5, np.float64)
    h = _handle(knnd, n, m, K, dtype="f64", precision="mixed")
    idx, key, flag = h.init_graph(_dev(pts), 5)
    h.sync()
    idx[7, 2] = n + 5
    idx[9, 0] = -3
    h.round(None, 5, 1, idx, key, flag)
    with pytest.raises(knnd.api._lib.KnndError) as e:
        h.sync()
    assert e.value.status == knnd.api._lib.KNND_EINVAL
    h.sync()  # cleared
    h.close()


@pytest.mark.parametrize("prec", PRECS)
def test_delta_proportion_stop_matches_oracle(knnd, prec):
    n, m, K, seed, S = 3000, 6, 10, 21, 2000
    pts = dirichlet_points(n, m, seed, np.float64)
    ref_full = oracle.build(pts, K, seed, S=S)
    delta = (ref_full["updates"][2] + 0.5) / (n * K)
    ref = oracle.build(pts, K, seed, S=S, stop_delta=delta)
    h = _handle(knnd, n, m, K, dtype="f64", precision=prec, fcc_samples=S, stop_delta=delta)
    out = h.build(_dev(pts), seed)
    h.close()
    assert out["rounds"] == ref["rounds"] == 3
    assert out["stop_reason"] == knnd.api._lib.KNND_STOP_DELTA
    assert out["updates"] == list(ref["updates"]) and out["fcc_hits"] == list(ref["hits"])
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m,K,dtype", [(2000, 6, 10, "f64"), (1500, 21, 20, "f32"), (800, 65, 32, "f32")])
def test_reverse_direction_lockstep(knnd, prec, n, m, K, dtype):
    # the variant comparator: x ranks y by D(y||x); every round against the oracle's
    pts = dirichlet_points(n, m, 23, np.float32 if dtype == "f32" else np.float64)
    assert _lockstep(knnd, pts, K, 23, prec, rounds=3, dtype=dtype, S=500, comparator="kl_reverse") <= max(2, n // 500)


def test_reverse_direction_build(knnd):
    # free-running: the three forms give the same graph, and the oracle's
    n, m, K, seed, S = 3000, 11, 12, 29, 2000
    pts = dirichlet_points(n, m, seed, np.float64)
    ref = oracle.build(pts, K, seed, S=S, comparator="kl_reverse")
    outs = {}
    for prec in PRECS:
        h = _handle(knnd, n, m, K, dtype="f64", precision=prec, fcc_samples=S, comparator="kl_reverse")
        outs[prec] = h.build(_dev(pts), seed)
        h.close()
    for prec, out in outs.items():
        assert out["rounds"] == ref["rounds"] and out["updates"] == list(ref["updates"]), prec
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"]), prec
        assert torch.equal(out["key"], outs["fp64"]["key"]), prec
    fwd = oracle.build(pts, K, seed, S=S)
    assert not np.array_equal(fwd["idx"], ref["idx"])  # the two directions rank differently


def _gauss(n, m, seed, dtype=np.float64):
    # any finite coordinates, both signs (the squared Euclidean comparator needs no simplex)
    return (np.random.default_rng(seed).standard_normal((n, m)) * 2.0).astype(dtype)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m,K,dtype,gauss", [(2000, 6, 10, "f64", True), (1500, 21, 20, "f32", True),
                                                 (800, 65, 32, "f32", False), (1200, 128, 17, "f64", True)])
def test_sqeuclidean_lockstep(knnd, prec, n, m, K, dtype, gauss):
    npdt = np.float32 if dtype == "f32" else np.float64
    pts = _gauss(n, m, 31, npdt) if gauss else dirichlet_points(n, m, 31, npdt)
    assert _lockstep(knnd, pts, K, 31, prec, rounds=3, dtype=dtype, S=500, comparator="sqeuclidean") <= max(2, n // 500)


def test_sqeuclidean_build(knnd):
    n, m, K, seed, S = 3000, 9, 12, 37, 2000
    pts = _gauss(n, m, seed)
    ref = oracle.build(pts, K, seed, S=S, comparator="sqeuclidean")
    outs = {}
    for prec in PRECS:
        h = _handle(knnd, n, m, K, dtype="f64", precision=prec, fcc_samples=S, comparator="sqeuclidean")
        outs[prec] = h.build(_dev(pts), seed)
        h.close()
    for prec, out in outs.items():
        assert out["rounds"] == ref["rounds"] and out["updates"] == list(ref["updates"]), prec
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"]), prec
        assert torch.equal(out["key"], outs["fp64"]["key"]), prec
    # recall against exact brute force: the metric comparator's neighbours are found
    q = np.arange(0, n, 15).astype(np.int32)
    bi, _ = oracle.bruteforce(pts, K, q, comparator="sqeuclidean")
    got = outs["mixed"]["idx"].cpu().numpy()
    rec = np.mean([len(set(bi[t]) & set(got[x])) / K for t, x in enumerate(q)])
    assert rec > 0.9, rec


def test_sqeuclidean_domain(knnd):
    n, m, K = 300, 4, 6
    pts = _gauss(n, m, 5)
    h = _handle(knnd, n, m, K, dtype="f64", precision="mixed", comparator="sqeuclidean")
    h.build(_dev(pts), 5)  # negative and zero coordinates are fine here
    bad = pts.copy()
    bad[7, 1] = np.nan
    with pytest.raises(knnd.api._lib.KnndError) as e:
        h.build(_dev(bad), 5)
    assert e.value.status == knnd.api._lib.KNND_EDOMAIN
    h.close()
    hk = _handle(knnd, n, m, K, dtype="f64", precision="mixed")  # KL needs coordinates > 0
    with pytest.raises(knnd.api._lib.KnndError) as e:
        hk.build(_dev(pts), 5)
    assert e.value.status == knnd.api._lib.KNND_EDOMAIN
    hk.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m,K,dtype,gauss", [(2000, 6, 10, "f64", True), (1500, 21, 20, "f32", True),
                                                 (800, 65, 32, "f32", False), (1000, 40, 40, "f64", True)])
def test_inner_product_lockstep(knnd, prec, n, m, K, dtype, gauss):
    # maximum inner product neighbours, key 0 - <x, y>: every round against the oracle's
    npdt = np.float32 if dtype == "f32" else np.float64
    pts = _gauss(n, m, 43, npdt) if gauss else dirichlet_points(n, m, 43, npdt)
    assert _lockstep(knnd, pts, K, 43, prec, rounds=3, dtype=dtype, S=500, comparator="inner") <= max(2, n // 500)


def test_inner_product_build(knnd):
    n, m, K, seed, S = 3000, 9, 12, 47, 2000
    pts = _gauss(n, m, seed)
    ref = oracle.build(pts, K, seed, S=S, comparator="inner")
    outs = {}
    for prec in PRECS:
        h = _handle(knnd, n, m, K, dtype="f64", precision=prec, fcc_samples=S, comparator="inner")
        outs[prec] = h.build(_dev(pts), seed)
        h.close()
    for prec, out in outs.items():
        assert out["rounds"] == ref["rounds"] and out["updates"] == list(ref["updates"]), prec
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"]), prec
        assert torch.equal(out["key"], outs["fp64"]["key"]), prec
    # the keys are -<x, y> (numpy, to the chain's rounding)
    idx = outs["mixed"]["idx"].cpu().numpy()
    key = outs["mixed"]["key"].cpu().numpy()
    ref_k = -(pts[:, None, :] * pts[idx]).sum(-1)
    assert np.allclose(key, ref_k, rtol=0, atol=1e-12 * np.abs(pts).sum(1).max() ** 2)


def test_bounded_wait_timeout_is_reported(knnd):
    # debug = 2: the tensor-core join's first tile waits on a barrier that no MMA
    # signals; the wait gives up after about a second, the call reports ETIMEOUT,
    # and the GPU context stays usable (no fault is involved)
    n, m, K, seed = 3000, 21, 20, 3
    pts = _dev(dirichlet_points(n, m, seed, np.float32))
    h = _handle(knnd, n, m, K, dtype="f32", precision="bf16x3", debug=2)
    with pytest.raises(knnd.api._lib.KnndError) as e:
        h.build(pts, seed)
    assert e.value.status == knnd.api._lib.KNND_ETIMEOUT
    h.close()
    h = _handle(knnd, n, m, K, dtype="f32", precision="bf16x3")
    out = h.build(pts, seed)
    h.close()
    ref = _handle(knnd, n, m, K, dtype="f32", precision="fp64")
    r = ref.build(pts, seed)
    ref.close()
    assert torch.equal(out["idx"], r["idx"])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("n,m,K", [(70000, 21, 20), (6000, 11, 32), (66000, 6, 8)])
@pytest.mark.parametrize("choice", [(1, 4, 0, "tma"), (4, 8, 3, "tma"), (16, 8, 1, "plain"), (2, 4, 5, "tma"),
                                    (8, 4, 0, "plain")])
def test_tuning_choices_same_graph(knnd, prec, n, m, K, choice):
    # the execution choices of the tuning table (round 1's split share, the
    # merge's per-lane keep, the TMA join's blocks per SM, the join's gathers)
    # change the speed only
    seed = 5
    pts = _dev(dirichlet_points(n, m, seed, np.float32))
    ref = _handle(knnd, n, m, K, dtype="f32", precision=prec)
    a = ref.build(pts, seed)
    ref.close()
    s, keep, blocks, form = choice
    h = _handle(knnd, n, m, K, dtype="f32", precision=prec, split_den=s, merge_keep=keep, join_blocks=blocks,
                    join_form=form)
    b = h.build(pts, seed)
    h.close()
    assert a["rounds"] == b["rounds"] and a["updates"] == b["updates"] and a["fcc_hits"] == b["fcc_hits"]
    assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["key"], b["key"])


def test_tuning_choices_batched_same_graphs(knnd):
    shapes = [(3000, 6, 8), (5000, 11, 16), (4000, 21, 32), (700, 21, 20)]
    pts = [_dev(dirichlet_points(n, m, 40 + i, np.float32)) for i, (n, m, K) in enumerate(shapes)]
    Ks = [K for _, _, K in shapes]
    seeds = [900 + i for i in range(len(shapes))]
    a = knnd.build_batched(pts, Ks, seeds)
    b = knnd.build_batched(pts, Ks, seeds, split_den=1, merge_keep=8, join_blocks=2, join_form="plain")
    for x, y in zip(a, b):
        assert x["rounds"] == y["rounds"] and x["updates"] == y["updates"]
        assert torch.equal(x["idx"], y["idx"]) and torch.equal(x["key"], y["key"])


@pytest.mark.parametrize("comparator", ["kl", "kl_reverse", "sqeuclidean"])
@pytest.mark.parametrize("n,m,K", [(20_000, 41, 16), (20_000, 60, 32), (30_000, 65, 20), (9_000, 70, 7),
                                   (5_001, 47, 31)])
def test_wide_tma_join_equals_fp64(knnd, comparator, n, m, K):
    # the TMA join of 41..72 coordinates (48, 64 or 72 padded; two columns per lane)
    # gives the FP64 form's graph bit for bit under every comparator, ragged item
    # tails and odd K included
    seed = 43
    pts = _gauss(n, m, seed, np.float32) if comparator == "sqeuclidean" else dirichlet_points(n, m, seed, np.float32)
    pts = _dev(pts)
    out = {}
    for prec in ("fp64", "mixed_tma"):
        h = _handle(knnd, n, m, K, dtype="f32", precision=prec, comparator=comparator)
        out[prec] = h.build(pts, seed)
        h.close()
    a, b = out["fp64"], out["mixed_tma"]
    assert b["join_kernel"] == "tma"
    assert a["rounds"] == b["rounds"] and a["updates"] == b["updates"] and a["fcc_hits"] == b["fcc_hits"]
    assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["key"], b["key"])
