"""The device-driven round loop (KNND_LOOP_GRAPH: one CUDA graph whose while
node runs the rounds, the stop rule applied on the device) against the host
loop (KNND_LOOP_HOST: one launch sequence and one stream synchronisation per
round).  Both must give the same graph, keys, flags and report, bit for bit:
for the stop on the clustering hits (Sec. 3.3), the delta rule and the round
cap, a complete initial graph, every precision and comparator, incremental
proposals, graph reuse across builds, recapture for new buffers, and the
host-memory build.
The free-running graph loop is also checked against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# the report fields fixed by the method; `rescored` and `merge_fallbacks` also
# depend on the order the join's atomics left each bucket in, and vary from run
# to run in either loop
KEYS = ("rounds", "stop_reason", "updates", "fcc_hits", "proposals", "init_pairs", "bound_violations",
        "join_survivors", "bound_audited")


@pytest.fixture(scope="module")
def knnd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2202_00517_gb300 as k
    return k


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _both(knnd, pts, K, seed, **kw):
    n, m = pts.shape
    dtype = "f32" if pts.dtype == torch.float32 else "f64"
    out = {}
    for loop in ("host", "graph"):
        h = knnd.Handle(n, m, K, dtype=dtype, loop=loop, **kw)
        out[loop] = h.build(pts, seed)
        h.close()
    return out["host"], out["graph"]


def _same(a, b):
    for k in KEYS:
        assert a[k] == b[k], k
    assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["key"], b["key"])
    assert torch.equal(a["flag"], b["flag"])


@pytest.mark.parametrize("prec", ["fp64", "mixed", "bf16x3"])
@pytest.mark.parametrize("comparator", ["kl", "kl_reverse", "sqeuclidean", "inner"])
def test_graph_loop_equals_host_loop(knnd, prec, comparator):
    pts = _dev(dirichlet_points(20_000, 21, 3, np.float32))
    a, b = _both(knnd, pts, 20, 3, precision=prec, comparator=comparator)
    assert a["rounds"] >= 3
    _same(a, b)


@pytest.mark.parametrize("kw,reason", [
    ({}, "KNND_STOP_FCC"),
    ({"max_rounds": 2}, "KNND_STOP_MAX_ROUNDS"),
    ({"stop_delta": None}, "KNND_STOP_DELTA"),  # set to stop after round 2
    ({"fcc_samples": 1}, None),          # one sample: the hits rarely rise, an early stop
    ({"incremental": True}, "KNND_STOP_FCC"),
])
def test_stop_reasons(knnd, kw, reason):
    n, m, K = 30_000, 11, 16
    pts = _dev(dirichlet_points(n, m, 5, np.float32))
    if "stop_delta" in kw:  # just above round 2's updates (which fall from round to round)
        full, _ = _both(knnd, pts, K, 5, precision="mixed")
        assert full["rounds"] > 2 and full["updates"][0] > full["updates"][1]
        kw = {"stop_delta": (full["updates"][1] + 0.5) / (n * K)}
    a, b = _both(knnd, pts, K, 5, precision="mixed", **kw)
    if reason:
        assert a["stop_reason"] == getattr(knnd.api._lib, reason)
    _same(a, b)


def test_complete_initial_graph(knnd):
    # n = K + 1: the initial graph is already complete, round 1 makes no update
    n, m, K = 17, 4, 16
    pts = _dev(dirichlet_points(n, m, 9, np.float64))
    a, b = _both(knnd, pts, K, 9, precision="fp64", fcc_samples=50)
    assert a["updates"][0] == 0 and a["rounds"] == 1
    _same(a, b)


def test_graph_reuse_and_recapture(knnd):
    # one handle: builds with the same buffers reuse the captured graph (new seed,
    # new points), new buffers recapture it; each equals a fresh host-loop build
    n, m, K = 25_000, 21, 20
    h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="graph")
    idx, key, flag = h.new_graph()
    runs = [(dirichlet_points(n, m, s, np.float32), s) for s in (11, 12)]
    got = []
    for p, s in runs:
        out = h.build(_dev(p), s, idx, key, flag)
        got.append({k: (v.clone() if torch.is_tensor(v) else v) for k, v in out.items()})
    got.append(h.build(_dev(runs[0][0]), runs[0][1]))  # fresh buffers
    launches = h.stats()["kernel_launches"]
    h.close()
    for (p, s), g in zip(runs + [runs[0]], got):
        ref = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="host")
        r = ref.build(_dev(p), s)
        ref.close()
        _same(r, g)
    assert launches > 0


def test_host_memory_build(knnd):
    n, m, K = 20_000, 11, 16
    p = torch.from_numpy(dirichlet_points(n, m, 13, np.float32))
    out = {}
    for loop in ("host", "graph"):
        h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop=loop)
        out[loop] = h.build_host(p.pin_memory(), 13)
        out[loop]["again"] = h.build_host(p.pin_memory(), 14)
        h.close()
    for k in KEYS:
        assert out["host"][k] == out["graph"][k], k
        assert out["host"]["again"][k] == out["graph"]["again"][k], k
    assert torch.equal(out["host"]["idx"], out["graph"]["idx"])
    assert torch.equal(out["host"]["key"], out["graph"]["key"])


def test_graph_loop_matches_oracle(knnd):
    n, m, K, seed, S = 3000, 6, 10, 17, 2000
    pts = dirichlet_points(n, m, seed, np.float64)
    ref = oracle.build(pts, K, seed, S=S)
    h = knnd.Handle(n, m, K, dtype="f64", precision="mixed", fcc_samples=S, loop="graph")
    out = h.build(_dev(pts), seed)
    h.close()
    assert out["rounds"] == ref["rounds"]
    assert out["updates"] == list(ref["updates"]) and out["fcc_hits"] == list(ref["hits"])
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])


def test_graph_loop_reports_device_errors(knnd):
    # a coordinate out of the domain is caught by the prepare step before any round
    n, m, K = 1000, 6, 10
    pts = dirichlet_points(n, m, 19, np.float64)
    pts[7, 2] = -1.0
    h = knnd.Handle(n, m, K, dtype="f64", precision="mixed", loop="graph")
    with pytest.raises(knnd.api._lib.KnndError):
        h.build(_dev(pts), 19)
    good = dirichlet_points(n, m, 19, np.float64)
    out = h.build(_dev(good), 19)  # the handle stays usable
    h.close()
    assert out["rounds"] >= 1


@pytest.mark.parametrize("n,m,K,kw", [
    (3, 2, 2, {}),                      # the smallest problem
    (500, 6, 10, {"max_rounds": 1}),    # one round: the cap stops it
    (2000, 6, 10, {"fcc_samples": 1}),
    (1500, 65, 33, {}),                 # K > 32
])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_edge_cases(knnd, n, m, K, kw, prec):
    pts = _dev(dirichlet_points(n, m, 21, np.float64))
    a, b = _both(knnd, pts, K, 21, precision=prec, **kw)
    _same(a, b)
    if kw.get("max_rounds") == 1:
        assert b["rounds"] == 1 and b["stop_reason"] in (knnd.api._lib.KNND_STOP_MAX_ROUNDS,
                                                          knnd.api._lib.KNND_STOP_FCC,
                                                          knnd.api._lib.KNND_STOP_ZERO)


def test_graph_loop_on_a_side_stream(knnd):
    # the graph is launched on the handle's stream, whatever stream captured it
    n, m, K = 5000, 11, 16
    pts = _dev(dirichlet_points(n, m, 23, np.float32))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="graph", stream=s)
        out = h.build(pts, 23)
        s.synchronize()
        h.close()
    ref = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="host")
    r = ref.build(pts, 23)
    ref.close()
    _same(r, out)
