// knnd_internal.cuh -- shared definitions of the CUDA translation units.
//
// Device data layout (one handle, n points, m coordinates padded to MP, a
// multiple of 8; padding coordinates are 0 in every table, so the padded
// terms of an fma chain are exact no-ops):
//   X64  n x MP  float64   the points
//   L64  n x MP  float64   log of the points
//   X32  n x MP  float32   the points rounded to FP32 (mixed form)
//   L32  n x MP  float32   log rounded to FP32 (mixed form)
//   negH n       float64   sum_i x_i log x_i (canonical fma chain)
//   nx   n       float64   sum_i |x_i|
//   cof_off n+1  int64     co-friend CSR offsets, cof n*K int32 entries
//   bucket       per point x, capacity K*K + (K+1)*indeg(x) at offset
//                K*K*x + (K+1)*cof_off[x]: the candidates the join emits for x.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/knnd.h"
#include "tune_table.h"

namespace knnd {

constexpr int kWarp = 32;

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and word streams with
// counter (c0, c1, c2, block); Lemire's bounded integers (ACM TOMACS 2019).
// --------------------------------------------------------------------------
struct Philox {
    uint32_t k0, k1, c0, c1, c2, block;
    uint32_t w[4];
    int pos;
    __device__ __forceinline__ Philox(uint64_t seed, uint32_t a, uint32_t b, uint32_t c)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0(a), c1(b), c2(c), block(0), pos(4) {}

    __device__ __forceinline__ void refill() {
        uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = block;
        uint32_t key0 = k0, key1 = k1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
            uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
            uint32_t n0 = hi1 ^ x1 ^ key0, n2 = hi0 ^ x3 ^ key1;
            x0 = n0;
            x1 = lo1;
            x2 = n2;
            x3 = lo0;
            key0 += 0x9E3779B9u;
            key1 += 0xBB67AE85u;
        }
        w[0] = x0;
        w[1] = x1;
        w[2] = x2;
        w[3] = x3;
        block += 1;
        pos = 0;
    }
    __device__ __forceinline__ uint32_t next() {
        if (pos == 4) refill();
        return w[pos++];
    }
    // uniform in [0, N), N >= 1
    __device__ __forceinline__ uint32_t bounded(uint32_t N) {
        uint32_t x = next();
        uint64_t prod = (uint64_t)x * N;
        uint32_t low = (uint32_t)prod;
        if (low < N) {
            uint32_t t = (0u - N) % N;
            while (low < t) {
                x = next();
                prod = (uint64_t)x * N;
                low = (uint32_t)prod;
            }
        }
        return (uint32_t)(prod >> 32);
    }
};

// Philox stream tags (counter word c2).
constexpr uint32_t kTagInit = 0;
constexpr uint32_t kTagFcc = 1;

// --------------------------------------------------------------------------
// Candidate order: (key ascending, index ascending).
// --------------------------------------------------------------------------
__device__ __forceinline__ bool lex_less(double ka, int ia, double kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Order-preserving 32-bit image of a float: a < b  <=>  sortable(a) < sortable(b)
// (unsigned), for every non-NaN a, b (-0 sorts just below +0).
__device__ __forceinline__ uint32_t sortable_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float from_sortable_bits(uint32_t s) {
    return __uint_as_float((s & 0x80000000u) ? (s & 0x7fffffffu) : ~s);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Status bits set by kernels in the device error word.
constexpr int kErrDomain = 1;
constexpr int kErrBucket = 2;
constexpr int kErrIndex = 4;
constexpr int kErrTimeout = 8;

// Instances sharing one handle (the batched form): the union of their
// graphs, whose arcs never cross instances, is processed as one graph with
// global point indices.  `of` == nullptr: a single instance covering [0, n).
struct InstView {
    const int32_t *of;      // global point -> instance
    const int64_t *base;    // instance -> its first global point
    const int32_t *n;       // instance -> its number of points
    const uint64_t *seed;   // instance -> its seed
    const int32_t *active;  // instance -> 1 while its rounds continue
    int64_t *cnt;           // instance -> kCntNum counters of the current round
    __device__ __forceinline__ int at(int64_t x) const { return of ? of[x] : 0; }
    __device__ __forceinline__ bool live(int64_t x) const { return !of || active[of[x]] != 0; }
};

// Hubs of one phase of a split round: phase 0 every hub; 1 the hubs whose
// index within their instance is below n_i / den; 2 the others.
__device__ __forceinline__ bool in_phase(const InstView &iv, int phase, int den, int64_t n, int64_t v)
{
    if (phase == 0) return true;
    int64_t local = v, ni = n;
    if (iv.of) {
        const int i = iv.of[v];
        local = v - iv.base[i];
        ni = iv.n[i];
    }
    return (local * den < ni) == (phase == 1);
}

// Per-row data the mixed join reads with every row it gathers, packed in one
// 16-byte record (one memory sector): the rejection threshold phi and the
// start of the row's bucket, K*K*x + (K+1)*cof_off[x].
struct __align__(16) RowMeta {
    float phi;
    int32_t pad;
    long long boff;
};

// State of the device-driven round loop (KNND_LOOP_GRAPH), in device memory:
// the round kernels read the seed and the round number from it, and the
// loop's last kernel records the round's counters and the stop decision.
struct LoopState {
    unsigned long long seed;
    int32_t round;        // rounds begun
    int32_t stop_reason;  // KNND_STOP_* once the loop has stopped, else 0
    long long updates[KNND_MAX_ROUNDS];
    long long hits[KNND_MAX_ROUNDS + 1];
    long long sums[5];  // rescored, bound violations, merge fallbacks, join survivors, audited pairs
};

// Device counters of one call (int64 each).
enum Counter : int {
    kCntUpdates = 0,
    kCntHits = 1,
    kCntRescored = 2,
    kCntBoundViol = 3,
    kCntFallback = 4,
    kCntSurvivors = 5,  // bucket entries the join wrote
    kCntAudited = 6,    // pairs checked by the bound audit (debug)
    kCntNum = 8
};

}  // namespace knnd

struct knnd_handle {
    int64_t n;
    int32_t m, MP, K;
    knnd_dtype dtype;
    knnd_precision prec;
    knnd_params prm;
    cudaStream_t stream;
    int device;
    int num_sms;
    int fail_alloc_at;  // > 0: the fail_alloc_at-th workspace allocation fails (KNND_TEST_FAIL_ALLOC)
    // execution choices for the current shape (params, else the tuning table)
    int split_den, merge_keep, join_blocks;
    int join_form;    // KNND_JOIN_TMA or KNND_JOIN_PLAIN (params, else the tuning table)
    int join_kernel;  // KNND_JOIN_*: the join the last launch_join ran
    int allocs;
    bool prepared;

    // precompute
    double *X64, *L64, *negH, *nx;
    float *X32, *L32;
    // per instance i, bits of non-negative doubles: [3i] max |log y_j|, [3i+1] max |negH|,
    // [3i+2] max sum_j |y_j| (the last two bound the reverse direction's FP32 errors)
    unsigned long long *smax_bits;
    int32_t *err;                   // device error word
    // reverse CSR
    int32_t *deg;     // n: in-degree; for the TMA join, |coF(v) \ F(v)| (those entries first in coF(v))
    int32_t *deg_mut; // n: for the TMA join, |coF(v) & F(v)| (those entries last in coF(v))
    int32_t *slot;    // n*K: each arc's position in its co-friend list
    // the mixed join's heavy hubs: items (hub, row group) and their count;
    // capacity nK/64 + 16 >= 2nK/256 + 2nK/1025 (rows over all hubs: 2nK)
    int2 *heavy_items;
    int32_t *heavy_nitems;
    int64_t *cof_off; // n+1
    int32_t *cof;     // n*K
    // incremental proposals (params.incremental): the new-flag of the arc x -> v
    // of every coF(v) entry; the flags knnd_build keeps when its caller passes
    // none; the flags of G_{r-1} during a round (NULL: every pair is proposed)
    uint8_t *cof_new;   // n*K
    uint8_t *flag_tmp;  // n*K
    const uint8_t *round_flag;
    bool csr_mutual;  // this round's CSR puts the mutual arcs apart (for the TMA join)
    int64_t *scan_tmp;
    int64_t scan_tmp_len;
    // per-row thresholds of the join filter
    double *tau;  // n: K-th key of the row
    int32_t *idxK;  // n: K-th index of the row
    knnd::RowMeta *meta;  // n: mixed form, rejection threshold and bucket start of each row
    double *Ex;   // n: mixed form, error bound of the FP32 dot
    // buckets
    int32_t *bcnt;  // n
    int64_t bucket_cap;
    // bucket entry: (sortable bits of u, index), u a float that orders the
    // candidates like their keys: mixed form u = -(FP32 dot), FP64 form
    // u = key rounded up to FP32.  FP64 form: the exact key at the same slot.
    int2 *bent;
    double *bkey;
    unsigned long long *join_queue;  // work-queue counters: [0] the TMA join's, [1] the merge's
    int32_t *fb_list;   // n: rows the merge's fast path leaves to its second kernel
    int32_t *fb_count;
    double *fb_T;       // n: the bound T of each such row's K-th key
    // counters
    int64_t *cnt;       // kCntNum device counters
    int64_t *cnt_host;  // pinned mirror
    // graph buffers for the host-memory build
    void *pts_dev;
    int64_t pts_dev_bytes;
    int32_t *idx_dev;
    double *key_dev;
    // the graph after the first phase of a split round (single instance only)
    int32_t *idxA;
    double *keyA;
    uint8_t *flagA;
    // per-phase CUDA-event timing (params.timing)
    static constexpr int kMaxPending = 256;
    cudaEvent_t ev[2 * kMaxPending];
    int pend_phase[kMaxPending];
    int npend;
    bool events_made;
    double phase_ms[KNND_NUM_PHASES];
    int64_t phase_count[KNND_NUM_PHASES];
    // batched form: instance tables (device) and their view
    int32_t ninst;
    knnd::InstView iv;
    int32_t *inst_of;
    int64_t *inst_base;
    int32_t *inst_n;
    uint64_t *inst_seed;
    int32_t *inst_active;
    int64_t *inst_cnt;
    // device-driven round loop (KNND_LOOP_GRAPH): state, pinned mirror, the
    // stream the round is captured on, the graph and the pointers it was
    // captured for, kernels of its first round and of each later round
    knnd::LoopState *loop_st;
    knnd::LoopState *loop_host;
    cudaStream_t cap_stream;
    cudaGraph_t loop_graph;
    cudaGraphExec_t loop_exec;
    const void *loop_for[3];
    int64_t loop_first_launches;
    int64_t loop_round_launches;
    // statistics
    int64_t launches;
    int64_t rounds_run;
    int64_t ws_bytes;
    double bound_c;  // c_m of the FP32 error bound
};

namespace knnd {

// ---- launch wrappers (each returns cudaGetLastError() of its launches) ----
cudaError_t launch_precompute(knnd_handle *h, const void *points, int64_t ld);
cudaError_t launch_precompute_from(knnd_handle *h, const void *points, int64_t ld, const void *const *ptrs,
                                   const int64_t *lds);
// round_dev: the round number is read on the device there (a device-driven loop), else `round`.
cudaError_t launch_fcc_batch(knnd_handle *h, const int32_t *idx, int32_t round, const int32_t *round_dev = nullptr);
cudaError_t launch_init_graph(knnd_handle *h, uint64_t seed, int32_t *idx, double *key, uint8_t *newflag);
cudaError_t launch_reverse_csr(knnd_handle *h, const int32_t *idx, const double *key);
cudaError_t launch_thresholds(knnd_handle *h, const int32_t *idx, const double *key);
// The join over the hubs [h_lo, h_hi) of phase `phase` (see in_phase, den = split_den).
cudaError_t launch_join(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase = 0,
                        int split_den = 1);
cudaError_t launch_join_tc(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase,
                           int split_den);
// The FP32 join with TMA-gathered rows and columns (join_tma.cu): the default
// mixed-form join where tma_join_supported(h) holds.
bool tma_join_supported(const knnd_handle *h);
// The join of the next launch_join is the TMA join (its rows skip the
// co-friends that are also friends: launch_reverse_csr puts them last in coF).
bool join_runs_tma(const knnd_handle *h);
cudaError_t launch_join_tma(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase,
                            int split_den);
double bound_c_bf16x3(int MP);
bool tc_supported(int MP, int K);
cudaError_t launch_merge(knnd_handle *h, int32_t *idx, double *key, uint8_t *newflag);
cudaError_t launch_merge_from(knnd_handle *h, const int32_t *in_idx, const double *in_key, const uint8_t *in_flag,
                              int32_t *idx, double *key, uint8_t *newflag, bool count);
cudaError_t launch_fcc(knnd_handle *h, const int32_t *idx, uint64_t seed, int32_t round, int64_t *hits_out,
                       const LoopState *loop = nullptr);  // loop: seed and round read from it on the device

// ---- handle set-up shared by the single-instance and batched forms ----
struct Caps {
    int64_t n;       // points
    int64_t tab;     // elements of each coordinate / log table (points x padded m)
    int64_t nK;      // arcs
    int64_t bucket;  // bucket entries
    int32_t ninst;   // instances (0: single-instance handle)
};
knnd_params default_params();
knnd_status make_handle(knnd_handle **out, const Caps &c, knnd_dtype dtype, knnd_precision precision,
                        const knnd_params &prm, void *stream);
void configure(knnd_handle *h, int64_t n, int32_t m, int32_t K);
void destroy_handle(knnd_handle *h);
knnd_status take_error(knnd_handle *h);
knnd_status round_ops(knnd_handle *h, uint64_t seed, int32_t round, int32_t *idx, double *key, uint8_t *newflag,
                      int64_t *fcc_hits);
knnd_status status_of(cudaError_t e);

// The tuning table's entry for a shape (kTuneDefault when none covers it).
inline TuneEntry tune_lookup(int MP, int K)
{
    for (const TuneEntry &t : kTuneTable)
        if (t.MP == MP && K >= t.K_lo && K <= t.K_hi) return t;
    return kTuneDefault;
}

// Range checks of the execution choices of knnd_params (0: from the table).
inline bool tuning_valid(const knnd_params &p)
{
    return p.split_den >= 0 && p.split_den <= 64 && (p.merge_keep == 0 || p.merge_keep == 4 || p.merge_keep == 8) &&
           p.join_blocks >= 0 && p.join_blocks <= 8 && p.join_form >= 0 && p.join_form <= KNND_JOIN_PLAIN;
}

inline int pad_coords(int m) {
    int mp = (m + 7) / 8 * 8;
    if (mp > 64 && mp <= 72) return 72;
    if (mp > 72 && mp <= 96) return 96;
    if (mp > 96) return 128;
    if (mp > 32 && mp <= 48) return 48;
    if (mp > 48 && mp <= 64) return 64;
    return mp;  // 8, 16, 24, 32
}

}  // namespace knnd
