// tune_table.h -- execution choices per shape class, written by
// paper_2202_00517_gb300/autotune.py from measurements on the device (see the
// comment block it writes below).  Each entry covers one padded coordinate
// count MP and a range of K; a shape no entry covers gets kTuneDefault.
//   split_den:   round 1 runs the hubs [0, n / split_den) first (1: one phase)
//   merge_keep:  candidates each lane of the merge's fast path keeps (4 or 8)
//   join_blocks: resident blocks per SM of the FP32 TMA join (0: as many as fit)
#pragma once

namespace knnd {

struct TuneEntry {
    int MP, K_lo, K_hi;
    int split_den, merge_keep, join_blocks;
};

constexpr TuneEntry kTuneDefault = {0, 0, 0, 8, 4, 0};

// Measured on NVIDIA GB300, 2026-12-04, by
//   python -m paper_2202_00517_gb300.autotune
// Per class: the workload, the fastest choice (split_den, merge_keep, join_blocks)
// with its time, and the default's time (CUDA events, best of two runs); the
// entry holds the fastest choice only when it beats the default by more than 1%.
constexpr TuneEntry kTuneTable[] = {
    // m = 6, K = 8: 117 instances of the mix's (m=6, K=8) class, batched; fastest (1, 4, 0) 24.84 ms, default 25.90 ms
    {8, 2, 12, 1, 4, 0},
    // m = 6, K = 16: 117 instances of the mix's (m=6, K=16) class, batched; fastest (4, 4, 0) 33.84 ms, default 33.94 ms
    {8, 13, 18, 8, 4, 0},
    // m = 6, K = 32: 105 instances of the mix's (m=6, K=32) class, batched; fastest (8, 4, 0) 73.62 ms, default 73.62 ms
    {8, 25, 32, 8, 4, 0},
    // m = 11, K = 8: 116 instances of the mix's (m=11, K=8) class, batched; fastest (1, 4, 0) 33.97 ms, default 35.50 ms
    {16, 2, 12, 1, 4, 0},
    // m = 11, K = 16: 109 instances of the mix's (m=11, K=16) class, batched; fastest (4, 4, 0) 40.73 ms, default 40.83 ms
    {16, 13, 18, 8, 4, 0},
    // m = 11, K = 32: 114 instances of the mix's (m=11, K=32) class, batched; fastest (8, 4, 4) 78.24 ms, default 78.31 ms
    {16, 25, 32, 8, 4, 0},
    // m = 21, K = 8: 113 instances of the mix's (m=21, K=8) class, batched; fastest (1, 4, 0) 41.05 ms, default 42.79 ms
    {24, 2, 12, 1, 4, 0},
    // m = 21, K = 16: 111 instances of the mix's (m=21, K=16) class, batched; fastest (4, 4, 0) 35.01 ms, default 35.07 ms
    {24, 13, 18, 8, 4, 0},
    // m = 21, K = 32: 124 instances of the mix's (m=21, K=32) class, batched; fastest (8, 4, 3) 101.20 ms, default 101.33 ms
    {24, 25, 32, 8, 4, 0},
    // m = 21, K = 20: one instance, n=2e5, m=21, K=20; fastest (4, 4, 0) 12.11 ms, default 12.13 ms
    {24, 19, 24, 8, 4, 0},
    // m = 65, K = 32: one instance, n=2e5, m=65, K=32; fastest (8, 4, 0) 37.32 ms, default 37.32 ms
    {72, 25, 32, 8, 4, 0},
};

}  // namespace knnd
