"""Autotuner of the execution choices per shape class; writes csrc/tune_table.h.

The choices change the speed of a build, never its result (the tests build the
same graphs under every choice):
  split_den   round 1 first runs the hubs [0, n / split_den), 1 = one phase;
  merge_keep  candidates each lane of the merge's fast path keeps (4 or 8);
  join_blocks resident blocks per SM of the FP32 TMA join (0 = as many as fit);
  join_tma    1: the FP32 join gathers by TMA where that form applies, 0: plain loads.

Classes: the (m, K) classes of the 4,096-instance mix (m in {6, 11, 21},
K in {8, 16, 32}), the n = 1e6, d = 20, K = 20 shape and the n = 4e6, d = 64,
K = 32 shape.  Each class is measured on a workload of its own shape: for a mix
class, its instances of the mix (every 4th one; batched build, the form those
shapes run in); for the two large shapes, one instance of 2e5 points.  Every
choice is timed with CUDA events over two runs after one warm-up.  The fastest
choice goes into the table when it beats the default by more than MARGIN (1 %,
above the run-to-run spread of these timings); otherwise the class keeps the
default.  Both times are written beside each entry.

    python -m paper_2202_00517_gb300.autotune [--out PATH] [--quick]

Needs a GPU and the built library; run it on the device the table is for.
"""
from __future__ import annotations

import argparse
import ctypes
import datetime
import itertools
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2202_00517_gb300 import _lib  # noqa: E402
from paper_2202_00517_gb300.datagen import dirichlet_points, instance_mix  # noqa: E402

OUT = os.path.join(HERE, "csrc", "tune_table.h")
SPLITS = (1, 4, 8, 16)
KEEPS = (4, 8)
BLOCKS = (0, 4, 3)
DEFAULT = (8, 4, 0, 1)
MARGIN = 0.01


def pad_m(m: int) -> int:
    mp = (m + 7) // 8 * 8
    for lo, hi, v in ((32, 48, 48), (48, 64, 64), (64, 72, 72), (72, 96, 96), (96, 128, 128)):
        if lo < mp <= hi:
            return v
    return mp


def k_range(K: int):
    """The K values a class's table entry covers."""
    for lo, hi in ((2, 12), (13, 18), (19, 24), (25, 32), (33, 64)):
        if lo <= K <= hi:
            return lo, hi
    raise ValueError(K)


def time_batched(pts, Ks, seeds, choice, reps=2):
    """Milliseconds of one batched build of the instances under `choice`."""
    import torch
    lib = _lib.load()
    count = len(pts)
    arr = (_lib.knnd_instance * count)()
    outs = []
    for i, (p, k) in enumerate(zip(pts, Ks)):
        n, m = p.shape
        idx = torch.empty((n, k), dtype=torch.int32, device=p.device)
        key = torch.empty((n, k), dtype=torch.float64, device=p.device)
        outs.append((idx, key))
        arr[i] = _lib.knnd_instance(p.data_ptr(), p.stride(0), n, m, k, seeds[i], idx.data_ptr(), key.data_ptr())
    s, keep, blocks, tma = choice
    prm = _lib.knnd_params(10000, 64, 1, 0, 0, 0, 0.0, 0, 0, s, keep, blocks,
                           _lib.KNND_JOIN_TMA if tma else _lib.KNND_JOIN_PLAIN)
    b = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    st = ctypes.c_void_p(stream.cuda_stream)
    _lib.check(lib.knnd_batch_create(ctypes.byref(b), count, ctypes.cast(arr, ctypes.c_void_p), _lib.KNND_F32,
                                     _lib.KNND_PREC_MIXED_FP32, ctypes.byref(prm), 0, st), "knnd_batch_create")
    try:
        _lib.check(lib.knnd_batch_run(b, None), "knnd_batch_run")
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.check(lib.knnd_batch_run(b, None), "knnd_batch_run")
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        lib.knnd_batch_destroy(b)
    return best


def time_single(p, K, seed, choice, reps=2):
    import torch

    import paper_2202_00517_gb300 as knnd
    s, keep, blocks, tma = choice
    n, m = p.shape
    h = knnd.Handle(n, m, K, dtype="f32", precision="mixed", split_den=s, merge_keep=keep, join_blocks=blocks,
                    join_form="tma" if tma else "plain")
    idx, key, flag = h.new_graph(p.device)
    stream = torch.cuda.current_stream()
    try:
        h.build(p, seed, idx, key, flag)
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.build(p, seed, idx, key, flag)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        h.close()
    return best


def choices_for(mp: int, K: int, quick: bool):
    tma_ok = mp <= 32 and K <= 32
    if quick:
        return [DEFAULT, (4, 4, 0, 1), (8, 8, 0, 1), (8, 4, 0, 0)]
    out = []
    for s, keep in itertools.product(SPLITS, KEEPS):
        out += [(s, keep, b, 1) for b in (BLOCKS if tma_ok else (0,))]
        if tma_ok:
            out.append((s, keep, 0, 0))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--quick", action="store_true", help="three choices per class (a smoke run of this script)")
    args = ap.parse_args(argv)
    import torch
    dev = torch.device("cuda", 0)
    mix = instance_mix(4096, 5)
    results = []  # (mp, K, m, workload, {choice: ms})
    for m, K in itertools.product((6, 11, 21), (8, 16, 32)):
        sel = [i for i, (n, mm, k) in enumerate(mix) if mm == m and k == K][::4]
        pts = [torch.from_numpy(dirichlet_points(mix[i][0], m, 0x5EED0000 + i, np.float32)).to(dev) for i in sel]
        seeds = [0x5EED0000 + i for i in sel]
        times = {c: time_batched(pts, [K] * len(sel), seeds, c) for c in choices_for(pad_m(m), K, args.quick)}
        results.append((pad_m(m), K, m, f"{len(sel)} instances of the mix's (m={m}, K={K}) class, batched", times))
        print(m, K, min(times.items(), key=lambda t: t[1]), "default", times.get(DEFAULT), flush=True)
        del pts
        torch.cuda.empty_cache()
    for m, K, seed in ((21, 20, 1), (65, 32, 2)):
        p = torch.from_numpy(dirichlet_points(200_000, m, seed, np.float32)).to(dev)
        times = {c: time_single(p, K, seed, c) for c in choices_for(pad_m(m), K, args.quick)}
        results.append((pad_m(m), K, m, f"one instance, n=2e5, m={m}, K={K}", times))
        print(m, K, min(times.items(), key=lambda t: t[1]), "default", times.get(DEFAULT), flush=True)
        del p
        torch.cuda.empty_cache()
    write_table(args.out, results, torch.cuda.get_device_name(0))


def write_table(path, results, device):
    lines = [
        "// tune_table.h -- execution choices per shape class, written by",
        "// paper_2202_00517_gb300/autotune.py from measurements on the device (see the",
        "// comment block it writes below).  Each entry covers one padded coordinate",
        "// count MP and a range of K; a shape no entry covers gets kTuneDefault.",
        "//   split_den:   round 1 runs the hubs [0, n / split_den) first (1: one phase)",
        "//   merge_keep:  candidates each lane of the merge's fast path keeps (4 or 8)",
        "//   join_blocks: resident blocks per SM of the FP32 TMA join (0: as many as fit)",
        "//   join_tma:    1: the FP32 join gathers by TMA where that form applies; 0: plain loads",
        "#pragma once",
        "",
        "namespace knnd {",
        "",
        "struct TuneEntry {",
        "    int MP, K_lo, K_hi;",
        "    int split_den, merge_keep, join_blocks, join_tma;",
        "};",
        "",
        f"constexpr TuneEntry kTuneDefault = {{0, 0, 0, {DEFAULT[0]}, {DEFAULT[1]}, {DEFAULT[2]}, {DEFAULT[3]}}};",
        "",
        f"// Measured on {device}, {datetime.date.today().isoformat()}, by",
        "//   python -m paper_2202_00517_gb300.autotune",
        "// Per class: the workload, the fastest choice (split_den, merge_keep, join_blocks, join_tma)",
        "// with its time, and the default's time (CUDA events, best of two runs); the",
        f"// entry holds the fastest choice only when it beats the default by more than {MARGIN:.0%}.",
        "constexpr TuneEntry kTuneTable[] = {",
    ]
    for mp, K, m, workload, times in results:
        best, t = min(times.items(), key=lambda kv: kv[1])
        lo, hi = k_range(K)
        d = times.get(DEFAULT)
        pick = best if (d is None or t < d * (1.0 - MARGIN)) else DEFAULT
        lines.append(f"    // m = {m}, K = {K}: {workload}; fastest {best} {t:.2f} ms, default "
                     f"{'%.2f ms' % d if d is not None else 'not timed'}")
        lines.append(f"    {{{mp}, {lo}, {hi}, {pick[0]}, {pick[1]}, {pick[2]}, {pick[3]}}},")
    lines += ["};", "", "}  // namespace knnd", ""]
    with open(path, "w") as fh:
        fh.write("\n".join(lines))
    print("wrote", path)


if __name__ == "__main__":
    main()
