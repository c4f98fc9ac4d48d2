"""The batched form on the real 4,096-instance mix (n log-uniform in
[200, 50,000], m in {6, 11, 21}, K in {8, 16, 32}, Dirichlet(1) points,
instance i seeded 0x5EED0000 + i, shapes drawn from seed 5), against the
oracle's build (Sec. 3: initial graph, synchronous rounds, statistical stop) of
every 64th instance: same rounds, update counts and clustering hits, and the
same graph under the tie rule."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points, instance_mix
from parity_util import check_invariants, compare_graphs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

COUNT, EVERY = 4096, 64


def test_batched_mix_every_64th_instance_against_oracle():
    import paper_2202_00517_gb300 as knnd
    mix = instance_mix(COUNT, 5)
    seeds = [0x5EED0000 + i for i in range(COUNT)]
    with cf.ThreadPoolExecutor(16) as ex:
        host = list(ex.map(lambda a: dirichlet_points(a[1][0], a[1][1], seeds[a[0]], np.float32), enumerate(mix)))
    pts = [torch.from_numpy(hh).cuda() for hh in host]
    res = knnd.build_batched(pts, [k for _, _, k in mix], seeds)
    torch.cuda.synchronize()
    sel = list(range(0, COUNT, EVERY))
    assert len(sel) == 64

    def ref(i):
        n, m, k = mix[i]
        return oracle.build(host[i].astype(np.float64), k, seeds[i], S=10_000)

    refs = [ref(i) for i in sel]  # each oracle build runs its own OpenMP threads
    ties = 0
    shapes = set()
    for i, r in zip(sel, refs):
        n, m, k = mix[i]
        shapes.add((m, k))
        b = res[i]
        assert b["rounds"] == r["rounds"], (i, mix[i])
        assert b["updates"] == list(r["updates"]), (i, mix[i])
        assert b["fcc_hits"] == list(r["hits"]), (i, mix[i])
        gi, gk = b["idx"].cpu().numpy(), b["key"].cpu().numpy()
        check_invariants(gi, gk)
        ties += compare_graphs(host[i].astype(np.float64), gi, gk, r["idx"], r["key"])
    print(f"64 sampled instances of the mix: {len(shapes)} (m, K) classes, near-tie rows {ties}")
    assert len(shapes) == 9
    assert ties <= 8
