"""The oracle's pins must reject a wrong oracle.

Each case plants one plausible mistake in a copy of the oracle's C source:
- a changed random draw (Philox4x32-10, Lemire's bounded integers);
- a dropped term, wrong sign or transposed operand of a comparator's key (Sec. 2.2);
- a wrong tie order;
- a missing part of the candidate pool or a wrong co-friend list (Sec. 3.1, Sec. 4.2);
- a wrong new-flag, update or proposal count;
- a flaw in the initial graph (Sec. 3.2);
- a changed clustering sample or stop rule (Sec. 3.3, Table 1);
- a wrong brute-force K-NN (Sec. 2.3) or diameter (Sec. 4.3).

Mistakes that make the oracle loop forever or crash are left out: they cannot pass
the pins, but they would only slow this check down.

The copy is compiled in a scratch folder, and the oracle pin files run against it in
a child process.  Every mutant must make them fail, and the unchanged copy must pass.
The mistakes are planted on the CPU, in the copy only.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC_PATH = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["test_oracle_random.py", "test_oracle_key.py", "test_oracle_graph.py", "test_oracle_paper.py"]

# (name, text of oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("philox_multiplier_swapped", "uint64_t p0 = (uint64_t)ORC_PH_M0 * (uint64_t)c0;",
     "uint64_t p0 = (uint64_t)ORC_PH_M1 * (uint64_t)c0;"),
    ("philox_nine_rounds", "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    ("philox_key_bump_dropped", "k1 += ORC_PH_W1;", "k1 += 0u;"),
    ("philox_output_words_swapped", "out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;",
     "out[0] = c1; out[1] = c0; out[2] = c2; out[3] = c3;"),
    ("philox_key_bumped_before_round",
     "        uint32_t n0 = hi1 ^ c1 ^ k0;\n        uint32_t n1 = lo1;\n        uint32_t n2 = hi0 ^ c3 ^ k1;",
     "        k0 += ORC_PH_W0;\n        k1 += ORC_PH_W1;\n        uint32_t n0 = hi1 ^ c1 ^ k0;\n"
     "        uint32_t n1 = lo1;\n        uint32_t n2 = hi0 ^ c3 ^ k1;\n        k0 -= ORC_PH_W0;\n        k1 -= ORC_PH_W1;"),
    ("lemire_low_half", "return (uint32_t)(mprod >> 32);", "return (uint32_t)mprod % N;"),
    ("lemire_no_rejection", "while (low < thresh) {", "while (0 && low < thresh) {"),
    ("negH_term_dropped", "acc = fma(pts[y * m + i], l, acc);", "acc = l + acc;"),
    ("key_sign", "return off[x] - dot;", "return off[x] + dot;"),
    ("key_transposed", "for (int i = 0; i < m; ++i) dot = fma(pts[x * m + i], L[y * m + i], dot);",
     "for (int i = 0; i < m; ++i) dot = fma(pts[y * m + i], L[x * m + i], dot);"),
    ("reverse_not_swapped", "        x = y;\n        y = t;", "        (void)t;"),
    ("sqe_factor", "return (off[x] - 2.0 * dot) + off[y];", "return (off[x] - dot) + off[y];"),
    ("inner_uses_logs", "    if (orc_cmp == 3) {\n        for", "    if (orc_cmp == 99) {\n        for"),
    ("tie_break_reversed", "if (p->idx < q->idx) return -1;\n    if (p->idx > q->idx) return 1;",
     "if (p->idx < q->idx) return 1;\n    if (p->idx > q->idx) return -1;"),
    ("pool_no_cofriends",
     "for (int64_t q = cf->off[x]; q < cf->off[x + 1]; ++q) buf[len++] = cf->list[q]; /* co-friends */",
     "/* co-friends dropped */"),
    ("pool_no_friends_of_cofriends", "        for (int j = 0; j < K; ++j) buf[len++] = idx[(int64_t)w * K + j];\n",
     "        (void)w;\n"),
    ("pool_keeps_self", "if (buf[t] == (int32_t)x) continue;", "if (0) continue;"),
    ("cofriends_wrong_owner", "c->list[c->off[v] + fill[v]] = (int32_t)x;", "c->list[c->off[v] + fill[v]] = v;"),
    ("newflag_inverted", "newflag[x * K + t] = (uint8_t)(old ? 0 : 1);", "newflag[x * K + t] = (uint8_t)(old ? 1 : 0);"),
    ("updates_count_old", "updates += old ? 0 : 1;", "updates += old ? 1 : 0;"),
    ("proposals_miscounted", "props += (int64_t)K * K + (int64_t)(K + 1) * (cf.off[x + 1] - cf.off[x]);",
     "props += (int64_t)K * K + (int64_t)K * (cf.off[x + 1] - cf.off[x]);"),
    ("init_may_pick_self", "int32_t y = (int32_t)yp + ((int64_t)yp >= x ? 1 : 0);",
     "int32_t y = (int32_t)yp + ((int64_t)yp > x ? 1 : 0);"),
    ("init_unsorted", "qsort(c, (size_t)K, sizeof(orc_cand), orc_cand_cmp);", "/* unsorted */"),
    ("fcc_same_position", "int j = jp + (jp >= i ? 1 : 0);", "int j = jp + (jp > i ? 1 : 0);"),
    ("fcc_one_direction", "if (orc_is_friend(idx, K, y, z) || orc_is_friend(idx, K, z, y)) hits += 1;",
     "if (orc_is_friend(idx, K, y, z)) hits += 1;"),
    ("fcc_round_not_in_counter", "orc_stream_init(&st, seed, (uint32_t)s, (uint32_t)round, 1u);",
     "orc_stream_init(&st, seed, (uint32_t)s, 0u, 1u);"),
    ("stop_strict", "if (hits[r] <= hits[r - 1]) break;", "if (hits[r] < hits[r - 1]) break;"),
    ("delta_rule_ignores_K", "stop_delta * (double)n * (double)K) break;", "stop_delta * (double)n) break;"),
    ("bruteforce_keeps_self", "if (y == x) continue;", "if (0) continue;"),
    ("undirected_one_direction", "            raw[deg[y] + fill[y]++] = (int32_t)x;\n",
     "            raw[deg[y] + fill[y]++] = y;\n"),
    ("diameter_upper_bound", "if (best_hi < 0 || 2 * e < best_hi) best_hi = 2 * e;",
     "if (best_hi < 0 || e < best_hi) best_hi = e;"),
    ("bfs_ecc_off_by_one", "dist[w] = dist[v] + 1;", "dist[w] = dist[v] + (dist[v] > 0 ? 1 : 2);"),
    ("init_keys_swapped", "c[cnt].key = orc_key_from_tables(pts, L, negH, m, x, y);",
     "c[cnt].key = orc_key_from_tables(pts, L, negH, m, y, x);"),
    ("seed_words_swapped", "s->key[0] = (uint32_t)(seed & 0xffffffffu);\n    s->key[1] = (uint32_t)(seed >> 32);",
     "s->key[1] = (uint32_t)(seed & 0xffffffffu);\n    s->key[0] = (uint32_t)(seed >> 32);"),
    ("stream_block_not_advanced", "        s->block += 1;\n", "        s->block += 0;\n"),
    ("delta_rule_inclusive", "if (stop_delta > 0.0 && (double)updates[r - 1] < stop_delta",
     "if (stop_delta > 0.0 && (double)updates[r - 1] <= stop_delta"),
    ("stop_on_zero_ignored", "if (stop_on_zero && updates[r - 1] == 0) break;",
     "if (0 && stop_on_zero && updates[r - 1] == 0) break;"),
    ("hits0_round_one", "hits[0] = orc_fcc(idx, n, K, seed, 0, S);", "hits[0] = orc_fcc(idx, n, K, seed, 1, S);"),
    ("sqe_col_norm_dropped", "return (off[x] - 2.0 * dot) + off[y];", "return (off[x] - 2.0 * dot) + 0.0 * off[y];"),
    ("sqe_row_norm_dropped", "return (off[x] - 2.0 * dot) + off[y];", "return (0.0 - 2.0 * dot) + off[y];"),
    ("inner_offset_one", "            off[y] = 0.0;", "            off[y] = 1.0;"),
    ("fcc_i_range_short", "int i = (int)orc_bounded(&st, (uint32_t)K);", "int i = (int)orc_bounded(&st, (uint32_t)(K - 1));"),
    ("fcc_x_range_short", "int64_t x = orc_bounded(&st, (uint32_t)n);", "int64_t x = orc_bounded(&st, (uint32_t)(n / 2));"),
    ("bruteforce_never_first", "while (t > 0 && orc_cand_cmp(&e, &c[t - 1]) < 0) {",
     "while (t > 1 && orc_cand_cmp(&e, &c[t - 1]) < 0) {"),
    ("bruteforce_keeps_first_k", "if (len == K && orc_cand_cmp(&e, &c[K - 1]) >= 0) continue;",
     "if (len == K) continue;"),
    ("bfs_disconnected_ignored", "return tail == n ? ecc : -1;", "return ecc;"),
    ("diameter_lower_from_first_sweep_only", "if (e > best_lo) best_lo = e;", "if (t == 0 && e > best_lo) best_lo = e;"),
]


def _run_pins(base, name, old, new):
    """Copy the oracle package under base/name with one text replaced, then run
    the pin files against the copy.  Returns (exit code, output, imported file)."""
    src = open(SRC_PATH).read()
    d = os.path.join(base, name)
    pkg = os.path.join(d, "oracle")
    os.makedirs(pkg)
    for f in ("__init__.py", "oracle.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), pkg)
    with open(os.path.join(pkg, "oracle.c"), "w") as fh:
        fh.write(src.replace(old, new) if old else src)
    # the copy comes first on the path; the child runs from the copy's folder so
    # that the repository's own oracle package is not found before it
    env = dict(os.environ, PYTHONPATH=d + os.pathsep + ROOT, OMP_NUM_THREADS="4")
    # build the copy first: a mutant that does not compile must not count as rejected
    where = subprocess.run([sys.executable, "-c", "import oracle; oracle.build_oracle(); print(oracle.__file__)"],
                           cwd=d, env=env, capture_output=True, text=True).stdout.strip()
    p = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join(ROOT, "tests", f) for f in PINS],
                        "-x", "-q", "-m", "not gpu"], cwd=d, env=env, capture_output=True, text=True)
    return p.returncode, p.stdout + p.stderr, where


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(SRC_PATH).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, f"{name}: its text occurs {src.count(old)} times in oracle.c"
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    cases = [("unchanged", "", "")] + MUTANTS
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda c: _run_pins(base, *c), cases))
    return {c[0]: (r, os.path.join(base, c[0])) for c, r in zip(cases, res)}


def test_unchanged_copy_passes(outcomes):
    (rc, out, where), d = outcomes["unchanged"]
    assert where.startswith(d), f"the copy did not build or was not imported ({where!r})"
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_reject_mutant(outcomes, name):
    (rc, out, where), d = outcomes[name]
    assert where.startswith(d), f"the copy did not build or was not imported ({where!r})"
    # exit code 1: tests ran and one failed (2-5 would be an error of the harness)
    assert rc == 1, f"mutant {name} passed the pins (exit {rc}):\n{out[-2000:]}"
    assert "FAILED" in out
