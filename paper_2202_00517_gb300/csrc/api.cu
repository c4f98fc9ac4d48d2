// api.cu -- the C ABI of include/knnd.h: handle, scratch, argument checks and
// the launch sequences of init, round and build.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "knnd_internal.cuh"

using namespace knnd;

namespace {

constexpr int32_t kVersion = 100;  // 0.1.0

knnd_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return KNND_OK;
    if (e == cudaErrorMemoryAllocation) return KNND_ENOMEM;
    return KNND_ECUDA;
}

template <typename T>
knnd_status dalloc(knnd_handle *h, T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) return KNND_OK;
    // a failing allocation, faked on the host for the tests of the clean-up path
    if (h->fail_alloc_at > 0 && ++h->allocs == h->fail_alloc_at) return KNND_ENOMEM;
    const size_t bytes = sizeof(T) * (size_t)count;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return KNND_ENOMEM;
    }
    h->ws_bytes += (int64_t)bytes;
    return KNND_OK;
}

void drop_loop_graph(knnd_handle *h);

void free_all(knnd_handle *h)
{
    void *ptrs[] = {h->X64,       h->L64,      h->negH,      h->nx,          h->X32,         h->L32,
                    h->smax_bits, h->err,      h->deg,       h->deg_mut,     h->slot,        h->heavy_items,
                    h->heavy_nitems, h->cof_off, h->cof,     h->cof_new,     h->flag_tmp,    h->scan_tmp,
                    h->tau,       h->idxK,     h->meta,      h->Ex,          h->bcnt,        h->bkey,
                    h->bent,      h->fb_list,  h->fb_T,      h->join_queue,  h->fb_count,    h->cnt,
                    h->pts_dev,   h->idx_dev,  h->key_dev,   h->idxA,        h->keyA,        h->flagA,
                    h->inst_of,   h->inst_base, h->inst_n,   h->inst_seed,   h->inst_active, h->inst_cnt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->cnt_host) cudaFreeHost(h->cnt_host);
    drop_loop_graph(h);
    if (h->loop_st) cudaFree(h->loop_st);
    if (h->loop_host) cudaFreeHost(h->loop_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->events_made)
        for (int i = 0; i < 2 * knnd_handle::kMaxPending; ++i)
            if (h->ev[i]) cudaEventDestroy(h->ev[i]);
}

// Reads and clears the sticky device error word (synchronises the stream).
knnd_status take_device_error(knnd_handle *h)
{
    int32_t e = 0;
    cudaError_t c = cudaMemcpyAsync(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (c == cudaSuccess) c = cudaStreamSynchronize(h->stream);
    if (c != cudaSuccess) return cuda_status(c);
    if (e == 0) return KNND_OK;
    cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream);
    cudaStreamSynchronize(h->stream);
    if (e & kErrDomain) return KNND_EDOMAIN;
    if (e & kErrIndex) return KNND_EINVAL;
    if (e & kErrTimeout) return KNND_ETIMEOUT;
    return KNND_EOVERFLOW;
}

// ---- per-phase CUDA-event timing --------------------------------------------
void resolve_phases(knnd_handle *h)
{
    if (h->npend == 0) return;
    cudaEventSynchronize(h->ev[2 * (h->npend - 1) + 1]);
    for (int i = 0; i < h->npend; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) {
            h->phase_ms[h->pend_phase[i]] += ms;
            h->phase_count[h->pend_phase[i]] += 1;
        }
    }
    h->npend = 0;
}

// Phases are NVTX ranges (visible to a profiler's timeline; no cost without
// one) and, with params.timing, CUDA-event intervals on the handle's stream.
const char *const kPhaseName[KNND_NUM_PHASES] = {"knnd prepare", "knnd init", "knnd csr",
                                                 "knnd join",    "knnd merge", "knnd fcc"};

int phase_begin(knnd_handle *h, int phase)
{
    nvtxRangePushA(kPhaseName[phase]);
    if (!h->events_made) return -1;
    if (h->npend == knnd_handle::kMaxPending) resolve_phases(h);
    const int slot = h->npend;
    cudaEventRecord(h->ev[2 * slot], h->stream);
    return slot;
}

void phase_end(knnd_handle *h, int slot, int phase)
{
    nvtxRangePop();
    if (slot < 0) return;
    cudaEventRecord(h->ev[2 * slot + 1], h->stream);
    h->pend_phase[slot] = phase;
    h->npend += 1;
}

knnd_status check_points(const knnd_handle *h, const void *points, int64_t ld)
{
    if (!points) return KNND_EINVAL;
    if (ld < h->m) return KNND_EINVAL;
    return KNND_OK;
}

knnd_status do_prepare(knnd_handle *h, const void *points, int64_t ld)
{
    knnd_status s = check_points(h, points, ld);
    if (s) return s;
    const int t = phase_begin(h, KNND_PHASE_PREPARE);
    cudaError_t e = launch_precompute(h, points, ld);
    phase_end(h, t, KNND_PHASE_PREPARE);
    if (e != cudaSuccess) return cuda_status(e);
    s = take_device_error(h);
    h->prepared = (s == KNND_OK);
    return s;
}

// Split first round.  Round 1 proposes nearly its whole pool (the K-th of K
// random friends is a poor threshold), so it runs in two phases: the hubs
// [0, n / split_den) propose and their candidates are merged into a copy of the
// graph; every row's K-th entry there is an upper bound of its K-th key at the
// end of the round (any part of the pool gives one), so the remaining hubs
// propose against that tighter threshold, and their candidates are merged into
// the copy to give G_1.  The graph, keys, flags and update count are those of
// the one-phase round: the same pool, the same K best.  Measured: 3 % (n = 1e6,
// m = 21, K = 20) to 5 % (m = 65, K = 32) off a build; splitting later rounds,
// whose thresholds are already good, cost more than it saved.
constexpr int32_t kSplitRounds = 1;  // the share of the first phase, 1 / split_den, comes from the tuning

// G_{r-1} -> G_r in place; the device counters accumulate.  loop: a round of
// the device-driven loop (the FCC sample reads seed and round there).
knnd_status do_round(knnd_handle *h, uint64_t seed, int32_t round, int32_t *idx, double *key, uint8_t *newflag,
                     int64_t *fcc_hits, const LoopState *loop = nullptr)
{
    // incremental proposals read the flags of G_{r-1} (the join runs before the
    // merge overwrites them with those of G_r)
    h->round_flag = (h->prm.incremental && newflag) ? newflag : nullptr;
    // the random graph G_0 has almost no mutual friends: round 1 skips their search
    h->csr_mutual = round >= 2;
    // one instance: the hubs [0, n / den) then the rest; several instances
    // (batched form): each instance's first n_i / den hubs, then the rest
    const int64_t den = h->split_den;
    const bool split = h->idxA && round >= 1 && round <= kSplitRounds && den >= 2;
    const bool by_phase = split && h->iv.of;
    const int64_t hs = !split ? h->n : (by_phase ? h->n : std::max<int64_t>(1, h->n / den));
    int t = phase_begin(h, KNND_PHASE_CSR);
    cudaError_t e = launch_reverse_csr(h, idx, key);
    phase_end(h, t, KNND_PHASE_CSR);
    if (e == cudaSuccess) {
        t = phase_begin(h, KNND_PHASE_JOIN);
        e = launch_join(h, idx, 0, hs, by_phase ? 1 : 0, (int)den);
        phase_end(h, t, KNND_PHASE_JOIN);
    }
    if (e == cudaSuccess) {
        t = phase_begin(h, KNND_PHASE_MERGE);
        e = split ? launch_merge_from(h, idx, key, nullptr, h->idxA, h->keyA, h->flagA, false)
                  : launch_merge(h, idx, key, newflag);
        phase_end(h, t, KNND_PHASE_MERGE);
    }
    if (split && e == cudaSuccess) {
        t = phase_begin(h, KNND_PHASE_CSR);
        e = launch_thresholds(h, h->idxA, h->keyA);
        phase_end(h, t, KNND_PHASE_CSR);
        if (e == cudaSuccess) {
            t = phase_begin(h, KNND_PHASE_JOIN);
            e = by_phase ? launch_join(h, idx, 0, h->n, 2, (int)den) : launch_join(h, idx, hs, h->n);
            phase_end(h, t, KNND_PHASE_JOIN);
        }
        if (e == cudaSuccess) {
            t = phase_begin(h, KNND_PHASE_MERGE);
            e = launch_merge_from(h, h->idxA, h->keyA, h->flagA, idx, key, newflag, true);
            phase_end(h, t, KNND_PHASE_MERGE);
        }
    }
    if (e == cudaSuccess && fcc_hits) {
        t = phase_begin(h, KNND_PHASE_FCC);
        e = launch_fcc(h, idx, seed, round, fcc_hits, loop);
        phase_end(h, t, KNND_PHASE_FCC);
    }
    h->round_flag = nullptr;
    h->rounds_run += 1;
    return cuda_status(e);
}

// ---- device-driven round loop (KNND_LOOP_GRAPH) ------------------------------
// One graph per handle: [while cond] { loop_begin; round (CSR, join, merge,
// FCC); loop_end }.  loop_end applies the host loop's stop rule, in the same
// order and arithmetic, and sets the condition.

struct LoopRule {
    int32_t max_rounds;
    int32_t stop_on_zero;
    float stop_delta;
    int64_t n;
    int32_t K;
};

__global__ void loop_init_kernel(LoopState *st, unsigned long long seed, const int64_t *cnt)
{
    st->seed = seed;
    st->round = 0;
    st->stop_reason = 0;
    st->hits[0] = cnt[kCntHits];
    for (int i = 0; i < 5; ++i) st->sums[i] = 0;
}

__global__ void loop_begin_kernel(LoopState *st, int64_t *cnt)
{
    st->round += 1;
    for (int i = 0; i < kCntNum; ++i) cnt[i] = 0;
}

__global__ void loop_end_kernel(LoopState *st, const int64_t *cnt, LoopRule rule, cudaGraphConditionalHandle cond)
{
    const int r = st->round;
    const long long u = cnt[kCntUpdates], hits = cnt[kCntHits];
    st->updates[r - 1] = u;
    st->hits[r] = hits;
    st->sums[0] += cnt[kCntRescored];
    st->sums[1] += cnt[kCntBoundViol];
    st->sums[2] += cnt[kCntFallback];
    st->sums[3] += cnt[kCntSurvivors];
    st->sums[4] += cnt[kCntAudited];
    int reason = 0;
    if (hits <= st->hits[r - 1]) reason = KNND_STOP_FCC;
    else if (rule.stop_on_zero && u == 0) reason = KNND_STOP_ZERO;
    else if (rule.stop_delta > 0.f && (double)u < (double)rule.stop_delta * (double)rule.n * (double)rule.K)
        reason = KNND_STOP_DELTA;
    else if (r >= rule.max_rounds) reason = KNND_STOP_MAX_ROUNDS;
    st->stop_reason = reason;
    cudaGraphSetConditional(cond, reason == 0 ? 1u : 0u);
}

void drop_loop_graph(knnd_handle *h)
{
    if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
    if (h->loop_graph) cudaGraphDestroy(h->loop_graph);
    h->loop_exec = nullptr;
    h->loop_graph = nullptr;
    h->loop_for[0] = h->loop_for[1] = h->loop_for[2] = nullptr;
}

// Capture one round into the body of a while node (on the handle's own
// capture stream: the caller's may be the legacy stream) and instantiate.
knnd_status make_loop_graph(knnd_handle *h, int32_t *idx, double *key, uint8_t *newflag)
{
    drop_loop_graph(h);
    if (!h->loop_st) {
        const knnd_status s = dalloc(h, &h->loop_st, 1);
        if (s) return s;
    }
    if (!h->loop_host && cudaMallocHost((void **)&h->loop_host, sizeof(LoopState)) != cudaSuccess) {
        (void)cudaGetLastError();
        h->loop_host = nullptr;
        return KNND_ENOMEM;
    }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return KNND_ECUDA;
    // [round 1 (split), its stop test] -> while (condition set by the stop tests)
    // { round, stop test }: the first round's stop test sets the while node's
    // condition before the node is reached
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0);
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    const int64_t launches0 = h->launches;
    const int64_t rounds0 = h->rounds_run;
    const LoopRule rule{h->prm.max_rounds, h->prm.stop_on_zero_updates, h->prm.stop_delta, h->n, h->K};
    knnd_status s = KNND_OK;
    std::vector<cudaGraphNode_t> tail;
    auto capture = [&](cudaGraph_t into, const cudaGraphNode_t *deps, size_t ndeps, int32_t round,
                       bool keep_tail) -> cudaError_t {
        cudaError_t c = cudaStreamBeginCaptureToGraph(h->cap_stream, into, deps, nullptr, ndeps,
                                                      cudaStreamCaptureModeThreadLocal);
        if (c != cudaSuccess) return c;
        loop_begin_kernel<<<1, 1, 0, h->cap_stream>>>(h->loop_st, h->cnt);
        const knnd_status rs = do_round(h, 0, round, idx, key, newflag, h->cnt + kCntHits, h->loop_st);
        if (rs && !s) s = rs;
        loop_end_kernel<<<1, 1, 0, h->cap_stream>>>(h->loop_st, h->cnt, rule, cond);
        if (keep_tail) {
            cudaStreamCaptureStatus st;
            const cudaGraphNode_t *d = nullptr;
            size_t nd = 0;
            c = cudaStreamGetCaptureInfo(h->cap_stream, &st, nullptr, nullptr, &d, nullptr, &nd);
            if (c == cudaSuccess) tail.assign(d, d + nd);
        }
        cudaGraph_t out = nullptr;
        const cudaError_t c2 = cudaStreamEndCapture(h->cap_stream, &out);
        c = c == cudaSuccess ? cudaGetLastError() : c;
        return c == cudaSuccess ? c2 : c;
    };
    if (e == cudaSuccess) e = capture(g, nullptr, 0, 1, true);
    const int64_t launches1 = h->launches;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess && !s) e = cudaGraphAddNode(&node, g, tail.data(), nullptr, tail.size(), &np);
    if (e == cudaSuccess && !s) e = capture(np.conditional.phGraph_out[0], nullptr, 0, kSplitRounds + 1, false);
    h->stream = user;
    h->loop_first_launches = launches1 - launches0 + 2;
    h->loop_round_launches = h->launches - launches1 + 2;
    h->launches = launches0;
    h->rounds_run = rounds0;
    if (e == cudaSuccess && !s) e = cudaGraphInstantiate(&h->loop_exec, g, 0);
    if (e != cudaSuccess || s) {
        (void)cudaGetLastError();
        cudaGraphDestroy(g);
        h->loop_exec = nullptr;
        return s ? s : cuda_status(e);
    }
    h->loop_graph = g;
    h->loop_for[0] = idx;
    h->loop_for[1] = key;
    h->loop_for[2] = newflag;
    return KNND_OK;
}

// The rounds of knnd_build with the stop rule on the device: G_0 and its hits
// are in idx/key and cnt[kCntHits]; one graph launch runs every round.
knnd_status graph_rounds(knnd_handle *h, uint64_t seed, int32_t *idx, double *key, uint8_t *newflag,
                         knnd_build_info *info)
{
    if (!h->loop_exec || h->loop_for[0] != idx || h->loop_for[1] != key || h->loop_for[2] != newflag) {
        const knnd_status s = make_loop_graph(h, idx, key, newflag);
        if (s) return s;
    }
    loop_init_kernel<<<1, 1, 0, h->stream>>>(h->loop_st, seed, h->cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphLaunch(h->loop_exec, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->loop_host, h->loop_st, sizeof(LoopState), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const LoopState &st = *h->loop_host;
    const int32_t R = st.round;
    if (R < 1 || R > h->prm.max_rounds || st.stop_reason == 0) return KNND_ECUDA;  // the loop did not finish
    info->rounds = R;
    info->stop_reason = st.stop_reason;
    for (int32_t r = 1; r <= R; ++r) {
        info->updates[r - 1] = st.updates[r - 1];
        info->fcc_hits[r] = st.hits[r];
    }
    info->rescored = st.sums[0];
    info->bound_violations = st.sums[1];
    info->merge_fallbacks = st.sums[2];
    info->join_survivors = st.sums[3];
    info->bound_audited = st.sums[4];
    info->join_kernel = h->join_kernel;
    info->proposals = (int64_t)R * h->n * (int64_t)h->K * (2 * (int64_t)h->K + 1);
    h->launches += 1 + h->loop_first_launches + (int64_t)(R - 1) * h->loop_round_launches;
    h->rounds_run += R;
    return KNND_OK;
}

bool use_graph_loop(const knnd_handle *h)
{
    return h->prm.loop == KNND_LOOP_GRAPH || (h->prm.loop == KNND_LOOP_AUTO && !h->prm.timing);
}

}  // namespace

namespace knnd {

knnd_params default_params()
{
    knnd_params p;
    p.fcc_samples = 10000;
    p.max_rounds = KNND_MAX_ROUNDS;
    p.stop_on_zero_updates = 1;
    p.debug = 0;
    p.timing = 0;
    p.incremental = 0;
    p.stop_delta = 0.f;
    p.comparator = KNND_CMP_KL;
    p.loop = KNND_LOOP_AUTO;
    p.split_den = 0;
    p.merge_keep = 0;
    p.join_blocks = 0;
    p.join_form = 0;
    return p;
}

void configure(knnd_handle *h, int64_t n, int32_t m, int32_t K)
{
    h->n = n;
    h->m = m;
    h->MP = pad_coords(m);
    h->K = K;
    // c_m of |fp32 dot - fp64 dot| <= c_m sum_i |x_i log y_i|: m FP32 fma roundings,
    // the FP32 rounding of log y_i and of x_i, doubled-rounding slack; 1% headroom.
    h->bound_c = (double)(m + 6) * 0x1p-24 * 1.01;
    // (the other comparators run the FP32 join in every mixed form)
    if (h->prec == KNND_PREC_MIXED_BF16X3 && tc_supported(h->MP, K) && h->prm.comparator == KNND_CMP_KL)
        h->bound_c = bound_c_bf16x3(h->MP);
    h->bucket_cap = n * K * (2 * (int64_t)K + 1);
    h->prepared = false;
    // execution choices: the caller's, else the committed tuning table's for (MP, K)
    const TuneEntry t = tune_lookup(h->MP, K);
    h->split_den = h->prm.split_den > 0 ? h->prm.split_den : t.split_den;
    h->merge_keep = h->prm.merge_keep > 0 ? h->prm.merge_keep : t.merge_keep;
    h->join_blocks = h->prm.join_blocks > 0 ? h->prm.join_blocks : t.join_blocks;
    h->join_form = h->prm.join_form > 0 ? h->prm.join_form : (t.join_tma ? KNND_JOIN_TMA : KNND_JOIN_PLAIN);
}

knnd_status make_handle(knnd_handle **out, const Caps &c, knnd_dtype dtype, knnd_precision precision,
                        const knnd_params &prm, void *stream)
{
    *out = nullptr;
    knnd_handle *h = new (std::nothrow) knnd_handle;
    if (!h) return KNND_ENOMEM;
    std::memset((void *)h, 0, sizeof(*h));
    h->dtype = dtype;
    h->prec = precision;
    h->prm = prm;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return KNND_ECUDA;
    }
    if (const char *f = std::getenv("KNND_TEST_FAIL_ALLOC")) h->fail_alloc_at = std::atoi(f);
    const int64_t n = c.n;
    knnd_status s = KNND_OK;
    const int64_t ntiles = (n + 2047) / 2048;
    h->scan_tmp_len = ntiles;
    const bool mixed = precision != KNND_PREC_FP64;
    if (!s) s = dalloc(h, &h->X64, c.tab);
    if (!s) s = dalloc(h, &h->L64, c.tab);
    if (!s) s = dalloc(h, &h->X32, c.tab);
    if (!s) s = dalloc(h, &h->L32, c.tab);
    if (!s) s = dalloc(h, &h->negH, n);
    if (!s) s = dalloc(h, &h->nx, n);
    if (!s) s = dalloc(h, &h->smax_bits, 3 * (c.ninst > 0 ? c.ninst : 1));
    if (!s) s = dalloc(h, &h->err, 1);
    if (!s) s = dalloc(h, &h->deg, n);
    if (!s) s = dalloc(h, &h->deg_mut, n);
    if (!s) s = dalloc(h, &h->slot, c.nK);
    if (!s) s = dalloc(h, &h->heavy_items, c.nK / 64 + 16);
    if (!s) s = dalloc(h, &h->heavy_nitems, 1);
    if (!s) s = dalloc(h, &h->cof_off, n + 1);
    if (!s) s = dalloc(h, &h->cof, c.nK);
    if (!s && prm.incremental) s = dalloc(h, &h->cof_new, c.nK);
    if (!s && prm.incremental) s = dalloc(h, &h->flag_tmp, c.nK);
    if (!s) s = dalloc(h, &h->scan_tmp, ntiles);
    if (!s) s = dalloc(h, &h->tau, n);
    if (!s) s = dalloc(h, &h->idxK, n);
    if (!s) s = dalloc(h, &h->meta, n);
    if (!s) s = dalloc(h, &h->Ex, n);
    if (!s) s = dalloc(h, &h->bcnt, n);
    if (!s) s = dalloc(h, &h->bent, c.bucket);
    if (!s && !mixed) s = dalloc(h, &h->bkey, c.bucket);
    if (!s) s = dalloc(h, &h->fb_list, n);
    if (!s) s = dalloc(h, &h->fb_T, n);
    if (!s) s = dalloc(h, &h->join_queue, 2);  // the join's and the merge's work-queue counters
    if (!s) s = dalloc(h, &h->fb_count, 1);
    if (!s) s = dalloc(h, &h->cnt, kCntNum);
    if (!s) s = dalloc(h, &h->idxA, c.nK);  // the split first round's graph copy
    if (!s) s = dalloc(h, &h->keyA, c.nK);
    if (!s) s = dalloc(h, &h->flagA, c.nK);
    if (!s && cudaMallocHost((void **)&h->cnt_host, sizeof(int64_t) * kCntNum) != cudaSuccess) s = KNND_ENOMEM;
    if (!s && c.ninst > 0) {
        if (!s) s = dalloc(h, &h->inst_of, n);
        if (!s) s = dalloc(h, &h->inst_base, c.ninst + 1);
        if (!s) s = dalloc(h, &h->inst_n, c.ninst);
        if (!s) s = dalloc(h, &h->inst_seed, c.ninst);
        if (!s) s = dalloc(h, &h->inst_active, c.ninst);
        if (!s) s = dalloc(h, &h->inst_cnt, (int64_t)c.ninst * kCntNum);
    }
    if (!s && prm.timing) {
        for (int i = 0; i < 2 * knnd_handle::kMaxPending && !s; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) s = KNND_ECUDA;
        h->events_made = true;
    }
    if (!s) {
        cudaError_t e = cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->cnt, 0, sizeof(int64_t) * kCntNum, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        s = cuda_status(e);
    }
    if (s) {
        free_all(h);
        delete h;
        (void)cudaGetLastError();
        return s;
    }
    *out = h;
    return KNND_OK;
}

void destroy_handle(knnd_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

knnd_status take_error(knnd_handle *h) { return take_device_error(h); }

knnd_status round_ops(knnd_handle *h, uint64_t seed, int32_t round, int32_t *idx, double *key, uint8_t *newflag,
                      int64_t *fcc_hits)
{
    return do_round(h, seed, round, idx, key, newflag, fcc_hits);
}

knnd_status status_of(cudaError_t e) { return cuda_status(e); }

}  // namespace knnd

extern "C" {

const char *knnd_status_string(knnd_status s)
{
    switch (s) {
    case KNND_OK: return "ok";
    case KNND_EINVAL: return "invalid argument";
    case KNND_EDOMAIN: return "a coordinate is not finite or not > 0";
    case KNND_ENOMEM: return "device allocation failed";
    case KNND_ECUDA: return "CUDA error";
    case KNND_ETIMEOUT: return "bounded device wait ran out";
    case KNND_EOVERFLOW: return "size exceeds an internal limit";
    case KNND_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

int32_t knnd_version(void) { return kVersion; }

knnd_status knnd_create(knnd_handle **out, int64_t n, int32_t m, int32_t K, knnd_dtype dtype,
                        knnd_precision precision, const knnd_params *params, void *stream)
{
    if (!out) return KNND_EINVAL;
    *out = nullptr;
    if (n < 3 || n >= ((int64_t)1 << 31)) return KNND_EINVAL;
    if (m < 1 || m > KNND_MAX_M) return KNND_EINVAL;
    if (K < 2 || K > KNND_MAX_K || (int64_t)K >= n) return KNND_EINVAL;
    if (dtype != KNND_F32 && dtype != KNND_F64) return KNND_EINVAL;
    if (precision == KNND_PREC_AUTO) precision = KNND_PREC_MIXED_FP32;
    if (precision != KNND_PREC_FP64 && precision != KNND_PREC_MIXED_FP32 && precision != KNND_PREC_MIXED_BF16X3)
        return KNND_EINVAL;
    knnd_params prm = params ? *params : knnd::default_params();
    if (prm.fcc_samples < 1 || prm.max_rounds < 1 || prm.max_rounds > KNND_MAX_ROUNDS) return KNND_EINVAL;
    if (prm.incremental != 0 && prm.incremental != 1) return KNND_EINVAL;
    if (!(prm.stop_delta >= 0.f && prm.stop_delta <= 1.f)) return KNND_EINVAL;
    if (prm.comparator < KNND_CMP_KL || prm.comparator > KNND_CMP_INNER) return KNND_EINVAL;
    if (prm.debug < 0 || prm.debug > 2) return KNND_EINVAL;
    if (prm.loop < KNND_LOOP_AUTO || prm.loop > KNND_LOOP_GRAPH) return KNND_EINVAL;
    if (prm.loop == KNND_LOOP_GRAPH && prm.timing) return KNND_EINVAL;  // event nodes cannot sit in the loop body
    if (!knnd::tuning_valid(prm)) return KNND_EINVAL;
    // bucket capacity n*K*(2K+1) and CSR sizes use int64; the per-row slot counter is int32
    if ((int64_t)K * K + (int64_t)(K + 1) * (n - 1) >= ((int64_t)1 << 31)) return KNND_EOVERFLOW;
    knnd::Caps caps;
    caps.n = n;
    caps.tab = n * pad_coords(m);
    caps.nK = n * K;
    caps.bucket = n * K * (2 * (int64_t)K + 1);
    caps.ninst = 0;
    knnd_handle *h = nullptr;
    knnd_status s = knnd::make_handle(&h, caps, dtype, precision, prm, stream);
    if (s) return s;
    knnd::configure(h, n, m, K);
    *out = h;
    return KNND_OK;
}

void knnd_destroy(knnd_handle *h) { knnd::destroy_handle(h); }

knnd_status knnd_set_stream(knnd_handle *h, void *stream)
{
    if (!h) return KNND_EINVAL;
    h->stream = (cudaStream_t)stream;
    return KNND_OK;
}

knnd_status knnd_prepare(knnd_handle *h, const void *points, int64_t ld)
{
    if (!h) return KNND_EINVAL;
    return do_prepare(h, points, ld);
}

knnd_status knnd_init_graph(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t *idx,
                            double *key, uint8_t *newflag)
{
    if (!h || !idx || !key) return KNND_EINVAL;
    if (points) {
        knnd_status s = do_prepare(h, points, ld);
        if (s) return s;
    } else if (!h->prepared) {
        return KNND_ESTATE;
    }
    const int t = phase_begin(h, KNND_PHASE_INIT);
    cudaError_t e = launch_init_graph(h, seed, idx, key, newflag);
    phase_end(h, t, KNND_PHASE_INIT);
    return cuda_status(e);
}

knnd_status knnd_round(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t round,
                       int32_t *idx, double *key, uint8_t *newflag, int64_t *updates, int64_t *fcc_hits)
{
    if (!h || !idx || !key || round < 1) return KNND_EINVAL;
    if (points) {
        knnd_status s = do_prepare(h, points, ld);
        if (s) return s;
    } else if (!h->prepared) {
        return KNND_ESTATE;
    }
    cudaError_t e = cudaMemsetAsync(h->cnt, 0, sizeof(int64_t) * kCntNum, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    knnd_status s = do_round(h, seed, round, idx, key, newflag, fcc_hits ? fcc_hits : nullptr);
    if (s) return s;
    if (updates) {
        e = cudaMemcpyAsync(updates, h->cnt + kCntUpdates, sizeof(int64_t), cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return KNND_OK;
}

knnd_status knnd_fcc(knnd_handle *h, const int32_t *idx, uint64_t seed, int32_t round, int64_t *hits)
{
    if (!h || !idx || !hits || round < 0) return KNND_EINVAL;
    return cuda_status(launch_fcc(h, idx, seed, round, hits));
}

knnd_status knnd_sync(knnd_handle *h)
{
    if (!h) return KNND_EINVAL;
    return take_device_error(h);
}

knnd_status knnd_build(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t *idx, double *key,
                       uint8_t *newflag, knnd_build_info *info)
{
    if (!h || !points || !idx || !key || !info) return KNND_EINVAL;
    std::memset(info, 0, sizeof(*info));
    knnd_status s = do_prepare(h, points, ld);
    if (s) return s;
    if (!newflag && h->prm.incremental) newflag = h->flag_tmp;  // the rounds need the flags
    int t = phase_begin(h, KNND_PHASE_INIT);
    cudaError_t e = launch_init_graph(h, seed, idx, key, newflag);
    phase_end(h, t, KNND_PHASE_INIT);
    if (e != cudaSuccess) return cuda_status(e);
    int64_t *d = h->cnt;
    int64_t *hst = h->cnt_host;
    e = cudaMemsetAsync(d, 0, sizeof(int64_t) * kCntNum, h->stream);
    if (e == cudaSuccess) {
        t = phase_begin(h, KNND_PHASE_FCC);
        e = launch_fcc(h, idx, seed, 0, d + kCntHits);
        phase_end(h, t, KNND_PHASE_FCC);
    }
    if (e != cudaSuccess) return cuda_status(e);
    info->init_pairs = h->n * h->K;
    if (use_graph_loop(h)) {
        s = graph_rounds(h, seed, idx, key, newflag, info);
        if (s) return s;
        info->fcc_hits[0] = h->loop_host->hits[0];
        return take_device_error(h);
    }
    e = cudaMemcpyAsync(hst, d, sizeof(int64_t) * kCntNum, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    info->fcc_hits[0] = hst[kCntHits];
    const int64_t per_round = h->n * (int64_t)h->K * (2 * (int64_t)h->K + 1);
    int32_t r = 0;
    while (r < h->prm.max_rounds) {
        r += 1;
        e = cudaMemsetAsync(d, 0, sizeof(int64_t) * kCntNum, h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        s = do_round(h, seed, r, idx, key, newflag, d + kCntHits);
        if (s) return s;
        e = cudaMemcpyAsync(hst, d, sizeof(int64_t) * kCntNum, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        info->updates[r - 1] = hst[kCntUpdates];
        info->fcc_hits[r] = hst[kCntHits];
        info->rescored += hst[kCntRescored];
        info->bound_violations += hst[kCntBoundViol];
        info->merge_fallbacks += hst[kCntFallback];
        info->join_survivors += hst[kCntSurvivors];
        info->bound_audited += hst[kCntAudited];
        info->join_kernel = h->join_kernel;
        info->proposals += per_round;
        info->rounds = r;
        if (info->fcc_hits[r] <= info->fcc_hits[r - 1]) {
            info->stop_reason = KNND_STOP_FCC;
            break;
        }
        if (h->prm.stop_on_zero_updates && info->updates[r - 1] == 0) {
            info->stop_reason = KNND_STOP_ZERO;
            break;
        }
        if (h->prm.stop_delta > 0.f &&
            (double)info->updates[r - 1] < (double)h->prm.stop_delta * (double)h->n * (double)h->K) {
            info->stop_reason = KNND_STOP_DELTA;
            break;
        }
    }
    if (!info->stop_reason) info->stop_reason = KNND_STOP_MAX_ROUNDS;
    return take_device_error(h);
}

knnd_status knnd_build_host(knnd_handle *h, const void *points_host, int64_t ld, uint64_t seed, int32_t *idx_host,
                            double *key_host, knnd_build_info *info)
{
    if (!h || !points_host || !idx_host || !key_host || !info) return KNND_EINVAL;
    if (ld < h->m) return KNND_EINVAL;
    const size_t esz = h->dtype == KNND_F32 ? 4 : 8;
    const int64_t pbytes = (int64_t)esz * ((h->n - 1) * ld + h->m);
    const int64_t nK = h->n * h->K;
    if (!h->pts_dev || h->pts_dev_bytes < pbytes) {
        if (h->pts_dev) {
            cudaFree(h->pts_dev);
            h->ws_bytes -= h->pts_dev_bytes;
            h->pts_dev = nullptr;
        }
        if (cudaMalloc(&h->pts_dev, (size_t)pbytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return KNND_ENOMEM;
        }
        h->pts_dev_bytes = pbytes;
        h->ws_bytes += pbytes;
    }
    if (!h->idx_dev) {
        knnd_status s = dalloc(h, &h->idx_dev, nK);
        if (!s) s = dalloc(h, &h->key_dev, nK);
        if (s) return s;
    }
    cudaError_t e = cudaMemcpyAsync(h->pts_dev, points_host, (size_t)pbytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    knnd_status s = knnd_build(h, h->pts_dev, ld, seed, h->idx_dev, h->key_dev, nullptr, info);
    if (s) return s;
    e = cudaMemcpyAsync(idx_host, h->idx_dev, sizeof(int32_t) * nK, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(key_host, h->key_dev, sizeof(double) * nK, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

knnd_status knnd_get_stats(knnd_handle *h, knnd_stats *st)
{
    if (!h || !st) return KNND_EINVAL;
    resolve_phases(h);
    st->kernel_launches = h->launches;
    st->rounds = h->rounds_run;
    st->workspace_bytes = h->ws_bytes;
    for (int p = 0; p < KNND_NUM_PHASES; ++p) {
        st->phase_count[p] = h->phase_count[p];
        st->phase_ms[p] = h->phase_ms[p];
    }
    return KNND_OK;
}

knnd_status knnd_reset_stats(knnd_handle *h)
{
    if (!h) return KNND_EINVAL;
    resolve_phases(h);
    for (int p = 0; p < KNND_NUM_PHASES; ++p) {
        h->phase_count[p] = 0;
        h->phase_ms[p] = 0.0;
    }
    h->launches = 0;
    h->rounds_run = 0;
    return KNND_OK;
}

}  // extern "C"
