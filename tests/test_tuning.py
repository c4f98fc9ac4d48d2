"""The committed tuning table (csrc/tune_table.h, written by the autotuner):
every entry is in range, entries do not overlap, and the table's reader in the
autotuner maps every benchmark class to one entry."""
import os
import re

from paper_2202_00517_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2202_00517_gb300", "csrc", "tune_table.h")


def _entries():
    text = open(TABLE).read()
    body = text[text.index("kTuneTable[]"):]
    rows = re.findall(r"^\s*\{(-?\d+), (-?\d+), (-?\d+), (-?\d+), (-?\d+), (-?\d+), (-?\d+)\},", body,
                      flags=re.M)
    return [tuple(int(v) for v in r) for r in rows]


def test_entries_in_range_and_disjoint():
    rows = _entries()
    assert rows
    seen = []
    for mp, lo, hi, s, keep, blocks, tma in rows:
        if hi < lo:  # an empty placeholder entry
            continue
        assert mp in (8, 16, 24, 32, 48, 64, 72, 96, 128)
        assert 2 <= lo <= hi <= 64
        assert 1 <= s <= 64 and keep in (4, 8) and 0 <= blocks <= 8 and tma in (0, 1)
        for mp2, lo2, hi2 in seen:
            assert mp2 != mp or hi2 < lo or hi < lo2, "overlapping entries"
        seen.append((mp, lo, hi))


def test_default_entry():
    text = open(TABLE).read()
    m = re.search(r"kTuneDefault = \{0, 0, 0, (\d+), (\d+), (\d+), (\d+)\}", text)
    assert m and tuple(int(v) for v in m.groups()) == autotune.DEFAULT


def test_class_ranges_cover_the_benchmark_shapes():
    for K in (8, 16, 20, 32):
        lo, hi = autotune.k_range(K)
        assert lo <= K <= hi
    assert autotune.pad_m(21) == 24 and autotune.pad_m(65) == 72 and autotune.pad_m(6) == 8
