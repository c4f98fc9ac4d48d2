"""Failure handling and resumption on the GPU, with no GPU fault:

* a workspace allocation that fails (faked on the host, KNND_TEST_FAIL_ALLOC)
  makes knnd_create return ENOMEM and frees everything it had allocated; a
  failing allocation of the graph loop's state makes that build return ENOMEM
  and leaves the handle usable;
* checkpoint / resume: the state at a round boundary is (idx, key, new-flags,
  round number, seed); rounds continued from a saved state on a fresh handle
  reproduce the uninterrupted run bit for bit (the random draws are keyed by
  seed, round and point).
"""
import os

import numpy as np
import pytest

from paper_2202_00517_gb300.datagen import dirichlet_points

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knnd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2202_00517_gb300 as k
    return k


def test_allocation_failure_frees_the_workspace(knnd):
    n, m, K = 50_000, 21, 20
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    try:
        for at in (1, 2, 5, 9, 14, 20):
            os.environ["KNND_TEST_FAIL_ALLOC"] = str(at)
            try:
                h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", timing=True)
            except knnd.api._lib.KnndError as e:
                assert e.status == knnd.api._lib.KNND_ENOMEM
                failures += 1
            else:
                h.close()
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert abs(free1 - free0) < (8 << 20), (at, free0 - free1)
    finally:
        os.environ.pop("KNND_TEST_FAIL_ALLOC", None)
    assert failures >= 5
    h = knnd.Handle(n, m, K, dtype="f32", precision="mixed")  # and the next one works
    h.close()


def test_loop_state_allocation_failure(knnd):
    # the graph loop allocates its state at the first build: a failure there is
    # ENOMEM from that build, and the next build on the same handle succeeds
    n, m, K, seed = 20_000, 11, 16, 3
    pts = torch.from_numpy(dirichlet_points(n, m, seed, np.float32)).cuda()
    h = None
    try:
        for at in range(1, 64):  # the first count create survives: its allocations + 1
            os.environ["KNND_TEST_FAIL_ALLOC"] = str(at)
            try:
                h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="graph")
                break
            except knnd.api._lib.KnndError as e:
                assert e.status == knnd.api._lib.KNND_ENOMEM
        assert h is not None
        with pytest.raises(knnd.api._lib.KnndError) as ei:
            h.build(pts, seed)
        assert ei.value.status == knnd.api._lib.KNND_ENOMEM
    finally:
        os.environ.pop("KNND_TEST_FAIL_ALLOC", None)
    out = h.build(pts, seed)
    h.close()
    ref = knnd.Handle(n, m, K, dtype="f32", precision="mixed", loop="host")
    r = ref.build(pts, seed)
    ref.close()
    assert out["rounds"] == r["rounds"] and out["updates"] == r["updates"]
    assert torch.equal(out["idx"], r["idx"]) and torch.equal(out["key"], r["key"])


@pytest.mark.parametrize("incremental", [False, True])
def test_resume_from_a_saved_round_matches_the_uninterrupted_run(knnd, incremental):
    n, m, K, seed, S = 40_000, 11, 16, 19, 5000
    pts = torch.from_numpy(dirichlet_points(n, m, seed, np.float32)).cuda()
    upd = torch.zeros(1, dtype=torch.int64, device="cuda")
    hits = torch.zeros(1, dtype=torch.int64, device="cuda")

    def rounds(h, idx, key, flag, r0, r1):
        log = []
        for r in range(r0, r1 + 1):
            h.round(None, seed, r, idx, key, flag, upd, hits)
            h.sync()
            log.append((int(upd.item()), int(hits.item())))
        return log

    # uninterrupted
    h = knnd.Handle(n, m, K, fcc_samples=S, incremental=incremental)
    idx, key, flag = h.init_graph(pts, seed)
    full = rounds(h, idx, key, flag, 1, 6)
    ref = (idx.cpu(), key.cpu(), flag.cpu())
    h.close()
    # three rounds, a checkpoint in host memory, a fresh handle, three more rounds
    h = knnd.Handle(n, m, K, fcc_samples=S, incremental=incremental)
    idx, key, flag = h.init_graph(pts, seed)
    first = rounds(h, idx, key, flag, 1, 3)
    saved = (idx.cpu(), key.cpu(), flag.cpu())
    h.close()
    h = knnd.Handle(n, m, K, fcc_samples=S, incremental=incremental)
    h.prepare(pts)
    idx, key, flag = (t.cuda() for t in saved)
    second = rounds(h, idx, key, flag, 4, 6)
    h.close()
    assert first + second == full
    assert torch.equal(idx.cpu(), ref[0]) and torch.equal(key.cpu(), ref[1]) and torch.equal(flag.cpu(), ref[2])
