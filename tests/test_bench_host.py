"""Host-side figures of the benchmark's CPU leg: the pair counts reported beside
the KL-evaluation metric.  The multiset is what a round scores (K^2 + (K+1)*indeg(x)
proposals per row, the per-point K + 2K^2 of the footnote in Sec. 4.4 on average);
the distinct pairs are the candidate pools of Sec. 3.1, enumerated here with
Python sets."""
import numpy as np

import bench
import oracle
from paper_2202_00517_gb300.datagen import dirichlet_points


def _pool_sets(idx, rows):
    n, K = idx.shape
    co = [[] for _ in range(n)]
    for x in range(n):
        for v in idx[x]:
            co[v].append(x)
    out = []
    for x in range(rows):
        s = set(idx[x]) | set(co[x])
        for v in idx[x]:
            s |= set(idx[v])
        for w in co[x]:
            s |= set(idx[w])
        s.discard(x)
        out.append(s)
    return out


def test_pair_counts_match_enumeration():
    n, m, K, seed, rows = 3000, 6, 10, 4, 500
    p = dirichlet_points(n, m, seed, np.float64)
    g, _ = oracle.init_graph(p, K, seed)
    c = bench.cpu_pair_counts(g, rows)
    _, _, _, _, props = oracle.round_(p, g, 0, rows)
    assert c["multiset"] == props
    assert c["unique"] == sum(len(s) for s in _pool_sets(g, rows))
    assert 0 < c["unique_fraction"] <= 1


def test_pair_trend_falls_as_the_graph_clusters():
    t = bench.cpu_pair_trend(6, 10, 4, n=3000)
    f = t["unique_fraction"]
    assert len(f) == t["rounds"] >= 2
    assert all(0 < x <= 1 for x in f)
    assert f[-1] < f[0]


def test_traffic_read_only_for_the_profiled_source(tmp_path, monkeypatch):
    # The roofline's DRAM traffic comes from a committed ncu summary, and only while
    # the join code it was taken on is the current one (its code hash recorded
    # there): a comment or layout edit keeps it, a code edit drops it.
    src = tmp_path / "paper_2202_00517_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "join.cu").write_text("// join v1\nint f() { return 1; }\n")
    sha = bench.code_sha256(str(src / "join.cu"))
    (tmp_path / "profiles" / "join_mixed_w.md").write_text(
        f"join.cu code sha256: {sha}\n\ndram bytes per full-size launch: 9.5e+09\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.join_traffic_per_launch("w") == 9.5e9
    assert bench.join_traffic_per_launch("other") is None
    (src / "join.cu").write_text("/* join\n   v2 */\nint  f()\n{ return 1; }  // same code\n")
    assert bench.join_traffic_per_launch("w") == 9.5e9
    (src / "join.cu").write_text("// join v1\nint f() { return 2; }\n")
    assert bench.join_traffic_per_launch("w") is None


def test_committed_profile_matches_the_join_source():
    # the benchmark workload's summary parses; its traffic is the join's, a few GB
    t = bench.join_traffic_per_launch("n1e6_d20_K20", "join_tma.cu", "join_tma")
    assert t is None or 1e9 < t < 1e11


def test_evaluation_count():
    # n K initial keys plus n (K + 2 K^2) proposals per round (Sec. 4.4 footnote)
    assert bench.evals_of(10, 2, 0) == 20
    assert bench.evals_of(10, 2, 3) == 20 + 3 * 10 * (2 + 8)


def test_l1_view_from_the_profiled_source(tmp_path, monkeypatch):
    # the L1 view divides the summary's wavefronts per launch by the run's launch time,
    # per SM and cycle, and is left out once the join code has changed
    src = tmp_path / "paper_2202_00517_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "join_tma.cu").write_text("int f() { return 1; }\n")
    sha = bench.code_sha256(str(src / "join_tma.cu"))
    (tmp_path / "profiles" / "join_tma_w.md").write_text(
        f"join_tma.cu code sha256: {sha}\n\nl1 data-pipe wavefronts per full-size launch: 3.0e+08\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    v = bench.join_l1_view("w", "join_tma.cu", "join_tma", 1e-3, 2000.0, 150)
    assert abs(v["achieved"] - 3.0e8 / (1e-3 * 2000e6 * 150)) < 1e-12 and v["peak"] == 1.0
    (src / "join_tma.cu").write_text("int f() { return 2; }\n")
    assert bench.join_l1_view("w", "join_tma.cu", "join_tma", 1e-3, 2000.0, 150) is None


def test_committed_profile_gives_the_l1_view():
    v = bench.join_l1_view("n1e6_d20_K20", "join_tma.cu", "join_tma", 2.9e-3, 2070.0, 152)
    assert v is None or 0.3 < v["achieved"] < 1.1
