// tune_table.h -- execution choices per shape class, written by
// paper_2202_00517_gb300/autotune.py from measurements on the device (see the
// comment block it writes below).  Each entry covers one padded coordinate
// count MP and a range of K; a shape no entry covers gets kTuneDefault.
//   split_den:   round 1 runs the hubs [0, n / split_den) first (1: one phase)
//   merge_keep:  candidates each lane of the merge's fast path keeps (4 or 8)
//   join_blocks: resident blocks per SM of the FP32 TMA join (0: as many as fit)
//   join_tma:    1: the FP32 join gathers by TMA where that form applies; 0: plain loads
#pragma once

namespace knnd {

struct TuneEntry {
    int MP, K_lo, K_hi;
    int split_den, merge_keep, join_blocks, join_tma;
};

constexpr TuneEntry kTuneDefault = {0, 0, 0, 8, 4, 0, 1};

// Measured on NVIDIA GB300, 2026-12-04, by
//   python -m paper_2202_00517_gb300.autotune
// Per class: the workload, the fastest choice (split_den, merge_keep, join_blocks, join_tma)
// with its time, and the default's time (CUDA events, best of two runs); the
// entry holds the fastest choice only when it beats the default by more than 1%.
constexpr TuneEntry kTuneTable[] = {
    // m = 6, K = 8: 117 instances of the mix's (m=6, K=8) class, batched; fastest (1, 4, 0, 0) 21.14 ms, default 22.60 ms
    {8, 2, 12, 1, 4, 0, 0},
    // m = 6, K = 16: 117 instances of the mix's (m=6, K=16) class, batched; fastest (8, 4, 0, 1) 26.24 ms, default 26.24 ms
    {8, 13, 18, 8, 4, 0, 1},
    // m = 6, K = 32: 105 instances of the mix's (m=6, K=32) class, batched; fastest (8, 8, 0, 1) 58.19 ms, default 59.01 ms
    {8, 25, 32, 8, 8, 0, 1},
    // m = 11, K = 8: 116 instances of the mix's (m=11, K=8) class, batched; fastest (1, 4, 0, 0) 28.94 ms, default 31.08 ms
    {16, 2, 12, 1, 4, 0, 0},
    // m = 11, K = 16: 109 instances of the mix's (m=11, K=16) class, batched; fastest (4, 4, 0, 1) 34.68 ms, default 34.73 ms
    {16, 13, 18, 8, 4, 0, 1},
    // m = 11, K = 32: 114 instances of the mix's (m=11, K=32) class, batched; fastest (8, 4, 0, 1) 66.43 ms, default 66.43 ms
    {16, 25, 32, 8, 4, 0, 1},
    // m = 21, K = 8: 113 instances of the mix's (m=21, K=8) class, batched; fastest (1, 4, 0, 1) 36.39 ms, default 38.16 ms
    {24, 2, 12, 1, 4, 0, 1},
    // m = 21, K = 16: 111 instances of the mix's (m=21, K=16) class, batched; fastest (8, 4, 0, 1) 31.17 ms, default 31.17 ms
    {24, 13, 18, 8, 4, 0, 1},
    // m = 21, K = 32: 124 instances of the mix's (m=21, K=32) class, batched; fastest (8, 4, 0, 0) 87.12 ms, default 89.01 ms
    {24, 25, 32, 8, 4, 0, 0},
    // m = 21, K = 20: one instance, n=2e5, m=21, K=20; fastest (4, 4, 0, 1) 11.34 ms, default 11.42 ms
    {24, 19, 24, 8, 4, 0, 1},
    // m = 65, K = 32: one instance, n=2e5, m=65, K=32; fastest (8, 4, 0, 1) 35.48 ms, default 35.48 ms
    {72, 25, 32, 8, 4, 0, 1},
};

}  // namespace knnd
