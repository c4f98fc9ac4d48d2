"""Comparison of a CUDA-path graph with the oracle's under the tie tolerance.

Both sides return, per point x, the K best candidates by (key, index).  The
CUDA path evaluates log with CUDA's double-precision log and the oracle with
the C library's, each within about one ulp, so two candidates whose FP64 keys
lie within rounding of each other may be ordered differently.  The rule: index
lists must be identical, except at rows where the oracle, re-keying the CUDA
path's entries itself, finds a sorted key vector equal to its own within
TOL_REL of the key scale |negH(x)| + |key| + 1; such rows are near-ties and are
counted.  Keys must agree within the same tolerance everywhere.  With the
reverse KL comparator (y ranked for x by D(y||x)) the offset negH belongs to
y, and the scale uses the largest |negH|; with the squared Euclidean one, the
largest |y|^2.
"""
import numpy as np

import oracle

TOL_REL = 1e-12


def compare_graphs(pts, gpu_idx, gpu_key, ref_idx, ref_key, rows=None, max_tie_rows=None, comparator="kl"):
    """Returns the number of near-tie rows; raises AssertionError on a real mismatch."""
    gpu_idx = np.asarray(gpu_idx)
    gpu_key = np.asarray(gpu_key)
    ref_idx = np.asarray(ref_idx)
    ref_key = np.asarray(ref_key)
    if rows is None:
        rows = np.arange(ref_idx.shape[0])
    K = ref_idx.shape[1]
    gi, gk, ri, rk = gpu_idx[rows], gpu_key[rows], ref_idx[rows], ref_key[rows]
    # key tolerance scale per row
    _, negH_all = oracle.logs(pts)
    if comparator == "kl":
        nh = np.abs(negH_all[rows])[:, None]
    elif comparator == "kl_reverse":  # the offset negH belongs to the candidate
        nh = np.full((len(rows), 1), np.abs(negH_all).max())
    else:  # squared Euclidean: the terms are |x|^2 and |y|^2
        sq = (np.asarray(pts) ** 2).sum(1)
        nh = np.full((len(rows), 1), sq.max())
    tol = TOL_REL * (2 * nh + np.abs(rk) + 1.0)
    bad = np.nonzero(np.any(gi != ri, axis=1))[0]
    ties = 0
    for b in bad:
        x = int(rows[b])
        ys = gi[b]
        assert len(set(ys.tolist())) == K and x not in ys.tolist(), f"row {x}: duplicate or self"
        kg = oracle.keys_pairs(pts, np.full(K, x), ys, comparator=comparator)
        assert np.all(np.abs(np.sort(kg) - rk[b]) <= tol[b]), (
            f"row {x}: CUDA list {ys.tolist()} vs oracle {ri[b].tolist()} is not a near-tie")
        ties += 1
    good = np.setdiff1d(np.arange(len(rows)), bad)
    assert np.all(np.abs(gk[good] - rk[good]) <= tol[good]), "keys differ beyond the tolerance"
    if max_tie_rows is not None:
        assert ties <= max_tie_rows, f"{ties} near-tie rows"
    return ties


def check_invariants(idx, key):
    """No self, no duplicate, rows sorted by (key, idx)."""
    idx = np.asarray(idx)
    key = np.asarray(key)
    n, K = idx.shape
    assert np.all(idx >= 0) and np.all(idx < n)
    assert np.all(idx != np.arange(n)[:, None])
    s = np.sort(idx, axis=1)
    assert np.all(s[:, 1:] != s[:, :-1])
    d = np.diff(key, axis=1)
    assert np.all((d > 0) | ((d == 0) & (idx[:, 1:] > idx[:, :-1])))
