"""The batched form (one launch per phase over many instances) against
separate builds of each instance and against the oracle.

Every instance must get exactly the graph, the rounds, the update counts and
the clustering hits that its own knnd_build gives (same seeds, same method);
a small workspace budget forces several sub-batches within one (m, K) class;
a sample of instances is also checked against the oracle's build.
"""
import numpy as np
import pytest

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    shapes = []
    for i in range(count):
        n = int(np.floor(40 * 50 ** rng.random()))
        m = int(rng.choice([2, 6, 11, 21]))
        K = int(rng.choice([2, 8, 16, 33]))
        K = min(K, n - 1)
        shapes.append((n, m, K))
    return shapes


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("limit", [0, 600_000])
def test_batched_equals_separate_builds(prec, limit):
    import paper_2202_00517_gb300 as knnd
    shapes = _mix(48, 3)
    pts = [torch.from_numpy(dirichlet_points(n, m, 1000 + i, np.float32)).cuda() for i, (n, m, K) in enumerate(shapes)]
    Ks = [K for _, _, K in shapes]
    seeds = [0x5EED0000 + i for i in range(len(shapes))]
    res = knnd.build_batched(pts, Ks, seeds, precision=prec, fcc_samples=700, workspace_limit=limit)
    for i, (n, m, K) in enumerate(shapes):
        h = knnd.Handle(n, m, K, dtype="f32", precision=prec, fcc_samples=700)
        ref = h.build(pts[i], seeds[i])
        h.close()
        b = res[i]
        assert b["rounds"] == ref["rounds"], i
        assert b["updates"] == ref["updates"] and b["fcc_hits"] == ref["fcc_hits"], i
        assert b["stop_reason"] == ref["stop_reason"], i
        assert torch.equal(b["idx"], ref["idx"]) and torch.equal(b["key"], ref["key"]), i


def test_batched_sample_against_oracle():
    import paper_2202_00517_gb300 as knnd
    shapes = [(300, 6, 8), (1200, 11, 16), (2000, 6, 10), (700, 21, 32), (64, 3, 5)]
    pts = [dirichlet_points(n, m, 77 + i, np.float64) for i, (n, m, K) in enumerate(shapes)]
    seeds = [11 * i + 5 for i in range(len(shapes))]
    res = knnd.build_batched([torch.from_numpy(p).cuda() for p in pts], [K for _, _, K in shapes], seeds,
                             fcc_samples=2000)
    for i, (n, m, K) in enumerate(shapes):
        ref = oracle.build(pts[i], K, seeds[i], S=2000)
        assert res[i]["rounds"] == ref["rounds"], i
        assert res[i]["updates"] == list(ref["updates"]), i
        assert res[i]["fcc_hits"] == list(ref["hits"]), i
        assert np.array_equal(res[i]["idx"].cpu().numpy(), ref["idx"]), i


def test_batched_rejects_bad_instances():
    import paper_2202_00517_gb300 as knnd
    from paper_2202_00517_gb300 import _lib
    p = torch.from_numpy(dirichlet_points(10, 4, 1, np.float32)).cuda()
    with pytest.raises(_lib.KnndError) as e:
        knnd.build_batched([p], [10], [1])  # K >= n
    assert e.value.status == _lib.KNND_EINVAL
    q = p.clone()
    q[3, 1] = -1.0
    with pytest.raises(_lib.KnndError) as e:
        knnd.build_batched([p, q], [3, 3], [1, 2])
    assert e.value.status == _lib.KNND_EDOMAIN


def test_batched_delta_stop_equals_separate_builds():
    import paper_2202_00517_gb300 as knnd
    shapes = _mix(24, 9)
    pts = [torch.from_numpy(dirichlet_points(n, m, 500 + i, np.float32)).cuda() for i, (n, m, K) in enumerate(shapes)]
    Ks = [K for _, _, K in shapes]
    seeds = [0x5EED0100 + i for i in range(len(shapes))]
    res = knnd.build_batched(pts, Ks, seeds, fcc_samples=700, stop_delta=0.02)
    reasons = set()
    for i, (n, m, K) in enumerate(shapes):
        h = knnd.Handle(n, m, K, dtype="f32", fcc_samples=700, stop_delta=0.02)
        ref = h.build(pts[i], seeds[i])
        h.close()
        b = res[i]
        assert b["rounds"] == ref["rounds"] and b["stop_reason"] == ref["stop_reason"], i
        assert b["updates"] == ref["updates"] and torch.equal(b["idx"], ref["idx"]), i
        reasons.add(b["stop_reason"])
    assert knnd.api._lib.KNND_STOP_DELTA in reasons


def test_batched_reverse_direction_equals_separate_builds():
    import paper_2202_00517_gb300 as knnd
    shapes = _mix(16, 12)
    pts = [torch.from_numpy(dirichlet_points(n, m, 700 + i, np.float32)).cuda() for i, (n, m, K) in enumerate(shapes)]
    Ks = [K for _, _, K in shapes]
    seeds = [0x5EED0200 + i for i in range(len(shapes))]
    res = knnd.build_batched(pts, Ks, seeds, fcc_samples=700, comparator="kl_reverse")
    for i, (n, m, K) in enumerate(shapes):
        h = knnd.Handle(n, m, K, dtype="f32", fcc_samples=700, comparator="kl_reverse")
        ref = h.build(pts[i], seeds[i])
        h.close()
        assert res[i]["rounds"] == ref["rounds"] and res[i]["updates"] == ref["updates"], i
        assert torch.equal(res[i]["idx"], ref["idx"]) and torch.equal(res[i]["key"], ref["key"]), i


def test_batched_sqeuclidean_equals_separate_builds():
    import paper_2202_00517_gb300 as knnd
    shapes = _mix(16, 14)
    rng = np.random.default_rng(8)
    pts = [torch.from_numpy(rng.standard_normal((n, m)).astype(np.float32)).cuda() for n, m, K in shapes]
    Ks = [K for _, _, K in shapes]
    seeds = [0x5EED0300 + i for i in range(len(shapes))]
    res = knnd.build_batched(pts, Ks, seeds, fcc_samples=700, comparator="sqeuclidean")
    for i, (n, m, K) in enumerate(shapes):
        h = knnd.Handle(n, m, K, dtype="f32", fcc_samples=700, comparator="sqeuclidean")
        ref = h.build(pts[i], seeds[i])
        h.close()
        assert res[i]["rounds"] == ref["rounds"] and res[i]["updates"] == ref["updates"], i
        assert torch.equal(res[i]["idx"], ref["idx"]) and torch.equal(res[i]["key"], ref["key"]), i


def test_batched_inner_product_equals_separate_builds():
    import paper_2202_00517_gb300 as knnd
    rng = np.random.default_rng(51)
    shapes = [(400, 6, 8), (900, 11, 16), (1500, 6, 8)]
    pts = [torch.from_numpy((rng.standard_normal((n, m)) * 2.0).astype(np.float32)).cuda() for n, m, _ in shapes]
    Ks = [k for _, _, k in shapes]
    seeds = [61, 62, 63]
    res = knnd.build_batched(pts, Ks, seeds, fcc_samples=700, comparator="inner")
    for (n, m, K), p, sd, r in zip(shapes, pts, seeds, res):
        h = knnd.Handle(n, m, K, dtype="f32", fcc_samples=700, comparator="inner")
        out = h.build(p, sd)
        h.close()
        assert out["rounds"] == r["rounds"] and out["updates"] == r["updates"]
        assert torch.equal(out["idx"], r["idx"]) and torch.equal(out["key"], r["key"])
