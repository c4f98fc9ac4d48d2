"""knnd_fcc_noalloc: the clustering sample for callers that cannot allocate.

Callers whose device memory is owned elsewhere (a memory pool or caching
allocator that holds nearly all of the GPU, a serving loop that forbids
allocation after start-up, a plug-in restricted to its host's allocator)
cannot create a knnd_handle, whose workspace knnd_create allocates.  The
no-allocation entry point gives them the stop test of their own descent loop.
Its scratch is a fixed device array inside the library, so two calls in a row
reuse it; both must return exactly what the handle-based knnd_fcc returns
(integer hit counts: equal, the tolerance of the parity tests for integers).

Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2202_00517_gb300.datagen import dirichlet_points

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _noalloc(lib, idx, seed, r, S, out):
    n, K = idx.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.knnd_fcc_noalloc(ctypes.c_void_p(idx.data_ptr()), n, K, seed, r, S,
                                ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_fcc_matches_handle_fcc_twice():
    assert torch.cuda.is_available()
    import paper_2202_00517_gb300 as knnd
    from paper_2202_00517_gb300 import _lib
    lib = _lib.load()
    n, m, K, seed, S = 20_000, 11, 16, 77, 10_000
    pts = torch.from_numpy(dirichlet_points(n, m, seed, np.float32)).cuda()
    h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", fcc_samples=S)
    idx, key, flag = h.init_graph(pts, seed)
    graphs = [idx.clone()]
    for r in (1, 2):
        h.round(None, seed, r, idx, key, flag)
        graphs.append(idx.clone())
    h.sync()
    ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    for r, g in enumerate(graphs):
        h.fcc(g, seed, r, ref)
        h.sync()
        for _ in range(2):  # two calls in a row share the fixed scratch array
            got.fill_(-7)
            assert _noalloc(lib, g, seed, r, S, got) == _lib.KNND_OK
            torch.cuda.synchronize()
            assert int(got.item()) == int(ref.item()), (r, int(got.item()), int(ref.item()))
    assert int(ref.item()) > 0
    h.close()


def test_noalloc_fcc_limits():
    from paper_2202_00517_gb300 import _lib
    lib = _lib.load()
    g = torch.zeros((100, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, g, 1, 0, _lib.KNND_NOALLOC_MAX_SAMPLES + 1, out) == _lib.KNND_EOVERFLOW
    assert _noalloc(lib, g, 1, 0, 0, out) == _lib.KNND_EINVAL
    assert lib.knnd_fcc_noalloc(None, 100, 4, 1, 0, 10, ctypes.c_void_p(out.data_ptr()), None) == _lib.KNND_EINVAL
    # largest accepted sample on a valid graph: the result is a count in [0, S]
    ring = ((torch.arange(100, device="cuda")[:, None] + torch.arange(1, 5, device="cuda")[None, :]) % 100)
    ring = ring.to(torch.int32).contiguous()
    S = _lib.KNND_NOALLOC_MAX_SAMPLES
    assert _noalloc(lib, ring, 1, 0, S, out) == _lib.KNND_OK
    torch.cuda.synchronize()
    # consecutive generators: every pair of friends is linked, so every sample hits
    assert int(out.item()) == S


def test_noalloc_fcc_bad_index_then_valid_graph():
    """A graph holding indices outside [0, n) gives hits = -1 (the kernel checks
    an index before following it, so nothing is read out of bounds); the error
    word lives in the shared scratch array, so the next call on a valid graph
    must clear it and return the handle's count again."""
    import paper_2202_00517_gb300 as knnd
    from paper_2202_00517_gb300 import _lib
    lib = _lib.load()
    n, K, seed, S = 1_000, 8, 5, 10_000
    ring = ((torch.arange(n, device="cuda")[:, None] + torch.arange(1, K + 1, device="cuda")[None, :]) % n)
    ring = ring.to(torch.int32).contiguous()
    bad = ring.clone()
    bad[0::2, :] = n        # every even row: only the index n, one past the last point
    bad[1::4, 0] = -1       # and some odd rows start with -1
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        out.fill_(123)
        assert _noalloc(lib, bad, seed, 3, S, out) == _lib.KNND_OK
        torch.cuda.synchronize()
        assert int(out.item()) == -1
    h = knnd.Handle(n, 4, K, dtype="f32", precision="mixed", fcc_samples=S)
    ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    h.fcc(ring, seed, 3, ref)
    h.sync()
    assert _noalloc(lib, ring, seed, 3, S, out) == _lib.KNND_OK
    torch.cuda.synchronize()
    assert int(out.item()) == int(ref.item()) == S  # consecutive generators: every sample hits
    h.close()
