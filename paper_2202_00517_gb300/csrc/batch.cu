// batch.cu -- the batched form: many independent instances (each its own
// points, m, K and seed) built together.  Instances with the same (m, K) form
// a class; a class is cut into sub-batches that fit the workspace budget.  A
// sub-batch is one union graph in global point indices -- its arcs never cross
// instances, so every pool of Sec. 3.1 stays inside one instance -- and runs
// through the same kernels as a single build: one launch per phase covers all
// its instances.  The initial graph and the clustering sample draw from each
// instance's own Philox streams over its local indices, and each instance
// keeps its own update and hit counters and its own stop decision (Sec. 3.3),
// taken on the device; a stopped instance's hubs and rows are skipped.  Every
// instance therefore gets exactly the graph, rounds and counts a separate
// knnd_build would give it.
//
// Execution.  Each sub-batch is one CUDA graph, captured at the first run and
// kept: the set-up, the initial graph, round 1 (split) and its stop test, then a
// conditional while node whose body is one round, the clustering sample and the
// per-instance stop test, whose last kernel keeps the loop going while any
// instance of the sub-batch is active; then the export of every instance's
// graph.  No host synchronisation happens inside a run.  Sub-batches are spread
// over up to kMaxSlots workspaces ("slots"), each with its own stream, so that
// up to kMaxSlots sub-batches run at once: the phases of one (the merge's FP64
// re-scores, the small per-round kernels, the tail of its last rounds) overlap
// the joins of another.  A slot runs its sub-batches in order; sub-batches go
// to slots largest first, each to the slot with the least work so far.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "knnd_internal.cuh"

using namespace knnd;

namespace {

constexpr int kMaxSlots = 4;

__global__ void fill_inst_of_kernel(const int64_t *__restrict__ base, int32_t ninst, int64_t n, int32_t *of)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    int lo = 0, hi = ninst - 1;  // last instance with base <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    of[x] = lo;
}

__global__ void set_ones_kernel(int32_t *a, int32_t n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 1;
}

struct History {
    int64_t *upd;       // ninst x max_rounds
    int64_t *hits;      // ninst x (max_rounds + 1)
    int64_t *rescored;  // ninst
    int64_t *fallback;  // ninst
    int32_t *rounds;    // ninst
    int32_t *reason;    // ninst
    int32_t *nactive;   // 1: instances still active after the current round
    int32_t *round;     // 1: the round the device-driven loop is in
};

__global__ void record_hits0_kernel(InstView iv, int32_t ninst, History hs, int32_t max_rounds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    hs.hits[(int64_t)i * (max_rounds + 1)] = iv.cnt[(int64_t)i * kCntNum + kCntHits];
}

// Start of a round of the loop: round number + 1, the instances' counters and
// the active count cleared.
__global__ void round_begin_kernel(History hs, int64_t *cnt, int32_t ninst)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (int64_t)ninst * kCntNum) cnt[t] = 0;
    if (t == 0) {
        *hs.round += 1;
        *hs.nactive = 0;
    }
}

// After round r: per-instance stop decision of Sec. 3.3 (iv) (hits of round r
// not above those of round r-1), or no update, or the round cap.
__global__ void stop_kernel(InstView iv, int32_t *active, int32_t ninst, History hs, int32_t max_rounds,
                            int32_t stop_on_zero, float stop_delta, int32_t K)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t r = *hs.round;
    if (i >= ninst || !active[i]) return;
    const int64_t *c = iv.cnt + (int64_t)i * kCntNum;
    const int64_t upd = c[kCntUpdates], hits = c[kCntHits];
    hs.upd[(int64_t)i * max_rounds + (r - 1)] = upd;
    int64_t *h = hs.hits + (int64_t)i * (max_rounds + 1);
    h[r] = hits;
    hs.rescored[i] += c[kCntRescored];
    hs.fallback[i] += c[kCntFallback];
    int reason = 0;
    if (hits <= h[r - 1]) reason = KNND_STOP_FCC;
    else if (stop_on_zero && upd == 0) reason = KNND_STOP_ZERO;
    else if (stop_delta > 0.f && (double)upd < (double)stop_delta * (double)iv.n[i] * (double)K) reason = KNND_STOP_DELTA;
    else if (r == max_rounds) reason = KNND_STOP_MAX_ROUNDS;
    if (reason) {
        active[i] = 0;
        hs.rounds[i] = r;
        hs.reason[i] = reason;
    } else {
        atomicAdd(hs.nactive, 1);
    }
}

// Last kernel of a round: the loop goes on while an instance is active.
__global__ void loop_cond_kernel(History hs, cudaGraphConditionalHandle cond)
{
    cudaGraphSetConditional(cond, *hs.nactive > 0 ? 1u : 0u);
}

// Global graph -> each instance's own arrays, indices made local.
__global__ void export_kernel(const int32_t *__restrict__ idx, const double *__restrict__ key, int64_t n, int K,
                              InstView iv, int32_t *const *out_idx, double *const *out_key)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int64_t x = e / K;
    const int t = (int)(e - x * K);
    const int i = iv.of[x];
    const int64_t b = iv.base[i];
    const int64_t o = (x - b) * K + t;
    out_idx[i][o] = idx[e] - (int32_t)b;
    out_key[i][o] = key[e];
}

// One sub-batch: its instances, their device tables (made once, at creation),
// its history and its CUDA graph.
struct SubBatch {
    int32_t m, K;
    std::vector<int32_t> members;  // indices into the instance array
    int64_t npts;
    double work;  // n K (2K + 1) summed: the pairs of one round
    int slot;
    int64_t *base;       // ninst + 1
    int32_t *n;
    uint64_t *seed;
    const void **ptrs;
    int64_t *lds;
    int32_t **oidx;
    double **okey;
    History hs;
    cudaGraphExec_t exec;
    int64_t launches_outer;  // kernels outside the loop body (set-up, round 1, export)
    int64_t launches_round;  // kernels of one round of the body
    int32_t join_kernel;     // KNND_JOIN_*: the join its rounds run
};

// A workspace and its stream: runs its sub-batches one after the other.
struct Slot {
    knnd_handle *h;  // sized for the largest of its sub-batches
    cudaStream_t stream;
    cudaEvent_t done;
    int32_t *idx;    // working graph
    double *key;
    std::vector<int> subs;
    double work;
};

}  // namespace

struct knnd_batch {
    std::vector<knnd_instance> inst;
    std::vector<SubBatch> subs;
    std::vector<Slot> slots;
    knnd_dtype dtype;
    knnd_precision prec;
    knnd_params prm;
    cudaStream_t stream;  // the caller's
    cudaEvent_t start;
    int64_t launches;
    int64_t ws_bytes;
};

namespace {

template <typename T>
knnd_status balloc(T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    if (cudaMalloc((void **)p, sizeof(T) * (size_t)count) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return KNND_ENOMEM;
    }
    return KNND_OK;
}

void free_sub(SubBatch &sb)
{
    if (sb.exec) cudaGraphExecDestroy(sb.exec);
    void *dev[] = {sb.base, sb.n, sb.seed, sb.ptrs, sb.lds, sb.oidx, sb.okey, sb.hs.upd, sb.hs.hits,
                   sb.hs.rescored, sb.hs.fallback, sb.hs.rounds, sb.hs.reason, sb.hs.nactive, sb.hs.round};
    for (void *p : dev)
        if (p) cudaFree(p);
}

void batch_free(knnd_batch *b)
{
    for (SubBatch &sb : b->subs) free_sub(sb);
    for (Slot &sl : b->slots) {
        if (sl.h) destroy_handle(sl.h);
        if (sl.idx) cudaFree(sl.idx);
        if (sl.key) cudaFree(sl.key);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (b->start) cudaEventDestroy(b->start);
    delete b;
}

// Device bytes one point of an instance with (m, K) needs in the workspace.
int64_t bytes_per_point(int32_t m, int32_t K, bool mixed, bool incremental)
{
    const int64_t MP = pad_coords(m);
    const int64_t bucket = (int64_t)K * (2 * K + 1) * (mixed ? 8 : 16);
    // tables, per-row scalars, buckets, CSR and arc slots, graph, the split round's graph copy (13 B per arc)
    return MP * 24 + 104 + bucket + (int64_t)K * (4 + 4 + 4 + 8 + 13 + (incremental ? 2 : 0));
}

// The sub-batch's device tables and history, filled once (synchronous copies).
knnd_status make_sub_tables(knnd_batch *b, SubBatch &sb)
{
    const int32_t ni = (int32_t)sb.members.size();
    const int32_t R = b->prm.max_rounds;
    knnd_status s = balloc(&sb.base, ni + 1);
    if (!s) s = balloc(&sb.n, ni);
    if (!s) s = balloc(&sb.seed, ni);
    if (!s) s = balloc(&sb.ptrs, ni);
    if (!s) s = balloc(&sb.lds, ni);
    if (!s) s = balloc(&sb.oidx, ni);
    if (!s) s = balloc(&sb.okey, ni);
    if (!s) s = balloc(&sb.hs.upd, (int64_t)ni * R);
    if (!s) s = balloc(&sb.hs.hits, (int64_t)ni * (R + 1));
    if (!s) s = balloc(&sb.hs.rescored, ni);
    if (!s) s = balloc(&sb.hs.fallback, ni);
    if (!s) s = balloc(&sb.hs.rounds, ni);
    if (!s) s = balloc(&sb.hs.reason, ni);
    if (!s) s = balloc(&sb.hs.nactive, 1);
    if (!s) s = balloc(&sb.hs.round, 1);
    if (s) return s;
    std::vector<int64_t> base(ni + 1), lds(ni);
    std::vector<int32_t> n(ni);
    std::vector<uint64_t> seed(ni);
    std::vector<const void *> ptrs(ni);
    std::vector<int32_t *> oidx(ni);
    std::vector<double *> okey(ni);
    int64_t off = 0;
    for (int32_t j = 0; j < ni; ++j) {
        const knnd_instance &in = b->inst[sb.members[j]];
        base[j] = off;
        n[j] = (int32_t)in.n;
        seed[j] = in.seed;
        ptrs[j] = in.points;
        lds[j] = in.ld;
        oidx[j] = in.idx;
        okey[j] = in.key;
        off += in.n;
    }
    base[ni] = off;
    cudaError_t e = cudaMemcpy(sb.base, base.data(), sizeof(int64_t) * (ni + 1), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.n, n.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.seed, seed.data(), sizeof(uint64_t) * ni, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.ptrs, ptrs.data(), sizeof(void *) * ni, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.lds, lds.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.oidx, oidx.data(), sizeof(int32_t *) * ni, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(sb.okey, okey.data(), sizeof(double *) * ni, cudaMemcpyHostToDevice);
    return status_of(e);
}

// Points the slot's handle at the sub-batch (its shape and instance tables).
void bind_sub(Slot &sl, const SubBatch &sb)
{
    knnd_handle *h = sl.h;
    configure(h, sb.npts, sb.m, sb.K);
    h->ninst = (int32_t)sb.members.size();
    h->iv.of = h->inst_of;
    h->iv.base = sb.base;
    h->iv.n = sb.n;
    h->iv.seed = sb.seed;
    h->iv.active = h->inst_active;
    h->iv.cnt = h->inst_cnt;
}

// Captures the sub-batch's whole build into one CUDA graph (on its slot's
// stream) and instantiates it:
//   set-up, precompute, initial graphs, hits of G_0;
//   round 1 (split), its sample and stop test, the loop condition;
//   while (an instance is active) { round, sample, stop test, condition };
//   export of each instance's graph.
knnd_status capture_sub(knnd_batch *b, SubBatch &sb)
{
    Slot &sl = b->slots[sb.slot];
    knnd_handle *h = sl.h;
    cudaStream_t st = sl.stream;
    bind_sub(sl, sb);
    const int32_t ni = (int32_t)sb.members.size();
    const int32_t R = b->prm.max_rounds;
    const int T = 256;
    const unsigned iblocks = (unsigned)((ni + T - 1) / T);
    const unsigned cblocks = (unsigned)(((int64_t)ni * kCntNum + T - 1) / T);
    uint8_t *flag = b->prm.incremental ? h->flag_tmp : nullptr;  // incremental proposals
    const int64_t l0 = h->launches;
    const int64_t r0 = h->rounds_run;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e) return status_of(e);
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0);
    knnd_status s = KNND_OK;
    std::vector<cudaGraphNode_t> tail;
    // one round of the loop: the round, the sample, the stop test, the condition
    auto round_body = [&](int32_t round) {
        round_begin_kernel<<<cblocks, T, 0, st>>>(sb.hs, h->inst_cnt, ni);
        const knnd_status rs = round_ops(h, 0, round, sl.idx, sl.key, flag, nullptr);
        if (rs && !s) s = rs;
        launch_fcc_batch(h, sl.idx, 0, sb.hs.round);
        stop_kernel<<<iblocks, T, 0, st>>>(h->iv, h->inst_active, ni, sb.hs, R, b->prm.stop_on_zero_updates,
                                           b->prm.stop_delta, sb.K);
        loop_cond_kernel<<<1, 1, 0, st>>>(sb.hs, cond);
        h->launches += 3;
    };
    auto end_capture = [&](cudaGraph_t into_out, bool keep_tail) -> cudaError_t {
        cudaError_t c = cudaGetLastError();
        if (keep_tail && c == cudaSuccess) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *d = nullptr;
            size_t nd = 0;
            c = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &d, nullptr, &nd);
            if (c == cudaSuccess) tail.assign(d, d + nd);
        }
        cudaGraph_t out = nullptr;
        const cudaError_t c2 = cudaStreamEndCapture(st, &out);
        (void)into_out;
        return c != cudaSuccess ? c : c2;
    };
    // set-up through round 1
    if (!e) e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (!e) {
        set_ones_kernel<<<iblocks, T, 0, st>>>(h->inst_active, ni);
        cudaMemsetAsync(sb.hs.rescored, 0, sizeof(int64_t) * ni, st);
        cudaMemsetAsync(sb.hs.fallback, 0, sizeof(int64_t) * ni, st);
        cudaMemsetAsync(sb.hs.upd, 0, sizeof(int64_t) * ni * R, st);
        cudaMemsetAsync(sb.hs.hits, 0, sizeof(int64_t) * ni * (R + 1), st);
        cudaMemsetAsync(sb.hs.round, 0, sizeof(int32_t), st);
        fill_inst_of_kernel<<<(unsigned)((sb.npts + T - 1) / T), T, 0, st>>>(sb.base, ni, sb.npts, h->inst_of);
        h->launches += 2;
        cudaError_t c = launch_precompute_from(h, nullptr, 0, sb.ptrs, sb.lds);
        if (!c) c = launch_init_graph(h, 0, sl.idx, sl.key, flag);
        if (!c) c = cudaMemsetAsync(h->inst_cnt, 0, sizeof(int64_t) * ni * kCntNum, st);
        if (!c) c = launch_fcc_batch(h, sl.idx, 0);
        if (c && !s) s = status_of(c);
        record_hits0_kernel<<<iblocks, T, 0, st>>>(h->iv, ni, sb.hs, R);
        h->launches += 1;
        round_body(1);
        e = end_capture(g, true);
    }
    const int64_t l1 = h->launches;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    if (!e && !s) e = cudaGraphAddNode(&wnode, g, tail.data(), nullptr, tail.size(), &np);
    // the loop body: rounds 2, 3, ... (single-phase rounds; the round number is read on the device)
    if (!e && !s) e = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (!e && !s) {
        round_body(2);
        e = end_capture(np.conditional.phGraph_out[0], false);
    }
    const int64_t l2 = h->launches;
    sb.join_kernel = h->join_kernel;
    // after the loop: every instance's graph to its own arrays
    if (!e && !s) e = cudaStreamBeginCaptureToGraph(st, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
    if (!e && !s) {
        const int64_t nK = sb.npts * sb.K;
        export_kernel<<<(unsigned)((nK + T - 1) / T), T, 0, st>>>(sl.idx, sl.key, sb.npts, sb.K, h->iv, sb.oidx,
                                                                  sb.okey);
        h->launches += 1;
        e = end_capture(g, false);
    }
    if (!e && !s) e = cudaGraphInstantiate(&sb.exec, g, 0);
    cudaGraphDestroy(g);
    sb.launches_outer = (l1 - l0) + (h->launches - l2);
    sb.launches_round = l2 - l1;
    h->launches = l0;
    h->rounds_run = r0;
    if (s) return s;
    if (e) {
        (void)cudaGetLastError();
        sb.exec = nullptr;
        return status_of(e);
    }
    return KNND_OK;
}

}  // namespace

extern "C" {

knnd_status knnd_batch_create(knnd_batch **out, int32_t count, const knnd_instance *inst, knnd_dtype dtype,
                              knnd_precision precision, const knnd_params *params, int64_t workspace_limit,
                              void *stream)
{
    if (!out) return KNND_EINVAL;
    *out = nullptr;
    if (count < 1 || !inst) return KNND_EINVAL;
    if (dtype != KNND_F32 && dtype != KNND_F64) return KNND_EINVAL;
    if (precision == KNND_PREC_AUTO) precision = KNND_PREC_MIXED_FP32;
    if (precision != KNND_PREC_FP64 && precision != KNND_PREC_MIXED_FP32 && precision != KNND_PREC_MIXED_BF16X3)
        return KNND_EINVAL;
    knnd_params prm = params ? *params : default_params();
    if (prm.fcc_samples < 1 || prm.max_rounds < 1 || prm.max_rounds > KNND_MAX_ROUNDS) return KNND_EINVAL;
    if (prm.incremental != 0 && prm.incremental != 1) return KNND_EINVAL;
    if (!(prm.stop_delta >= 0.f && prm.stop_delta <= 1.f)) return KNND_EINVAL;
    if (prm.comparator < KNND_CMP_KL || prm.comparator > KNND_CMP_INNER) return KNND_EINVAL;
    if (prm.loop < KNND_LOOP_AUTO || prm.loop > KNND_LOOP_GRAPH) return KNND_EINVAL;
    if (!tuning_valid(prm)) return KNND_EINVAL;
    prm.timing = 0;  // phase timing is a single-instance feature (events cannot sit in the loop body)
    const bool mixed = precision != KNND_PREC_FP64;
    for (int32_t i = 0; i < count; ++i) {
        const knnd_instance &in = inst[i];
        if (!in.points || !in.idx || !in.key) return KNND_EINVAL;
        if (in.n < 3 || in.n >= ((int64_t)1 << 31)) return KNND_EINVAL;
        if (in.m < 1 || in.m > KNND_MAX_M || in.ld < in.m) return KNND_EINVAL;
        if (in.K < 2 || in.K > KNND_MAX_K || (int64_t)in.K >= in.n) return KNND_EINVAL;
    }
    if (workspace_limit <= 0) workspace_limit = (int64_t)32 << 30;
    knnd_batch *b = new (std::nothrow) knnd_batch();
    if (!b) return KNND_ENOMEM;
    b->inst.assign(inst, inst + count);
    b->dtype = dtype;
    b->prec = precision;
    b->prm = prm;
    b->stream = (cudaStream_t)stream;
    // classes by (m, K); sub-batches within the budget, in input order
    std::map<std::pair<int32_t, int32_t>, std::vector<int32_t>> classes;
    for (int32_t i = 0; i < count; ++i) classes[{inst[i].m, inst[i].K}].push_back(i);
    int64_t largest = 0;  // bytes of the largest sub-batch
    for (auto &kv : classes) {
        const int32_t m = kv.first.first, K = kv.first.second;
        const int64_t bpp = bytes_per_point(m, K, mixed, prm.incremental != 0);
        SubBatch cur{};
        cur.m = m;
        cur.K = K;
        auto flush = [&]() {
            if (cur.members.empty()) return;
            largest = std::max(largest, cur.npts * bpp);
            b->subs.push_back(cur);
            cur = SubBatch{};
            cur.m = m;
            cur.K = K;
        };
        for (int32_t i : kv.second) {
            const int64_t ni = inst[i].n;
            const bool over = (cur.npts + ni) * bpp > workspace_limit ||
                              (int64_t)K * K + (int64_t)(K + 1) * (cur.npts + ni) >= ((int64_t)1 << 31);
            if (!cur.members.empty() && over) flush();
            cur.members.push_back(i);
            cur.npts += ni;
            cur.work += (double)ni * K * (2.0 * K + 1.0);
        }
        flush();
    }
    // slots: as many as sub-batches, at most kMaxSlots, and as many workspaces of the
    // largest sub-batch's size as 85 % of the free device memory holds
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        (void)cudaGetLastError();
        free_b = 0;
    }
    int nslots = std::min<int>(kMaxSlots, (int)b->subs.size());
    if (largest > 0) nslots = std::min<int64_t>(nslots, std::max<int64_t>(1, (int64_t)(0.85 * free_b) / largest));
    b->slots.resize(std::max(1, nslots));
    std::vector<int> order(b->subs.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->subs[x].work > b->subs[y].work; });
    for (int j : order) {  // largest first, to the least loaded slot
        int best = 0;
        for (int t = 1; t < (int)b->slots.size(); ++t)
            if (b->slots[t].work < b->slots[best].work) best = t;
        b->subs[j].slot = best;
        b->slots[best].work += b->subs[j].work;
        b->slots[best].subs.push_back(j);
    }
    knnd_status s = cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) == cudaSuccess ? KNND_OK : KNND_ECUDA;
    for (Slot &sl : b->slots) {
        if (s) break;
        std::sort(sl.subs.begin(), sl.subs.end());  // input order within a slot
        Caps caps = {0, 0, 0, 0, 0};
        for (int j : sl.subs) {
            const SubBatch &sb = b->subs[j];
            caps.n = std::max(caps.n, sb.npts);
            caps.tab = std::max(caps.tab, sb.npts * pad_coords(sb.m));
            caps.nK = std::max(caps.nK, sb.npts * sb.K);
            caps.bucket = std::max(caps.bucket, sb.npts * sb.K * (2 * (int64_t)sb.K + 1));
            caps.ninst = std::max(caps.ninst, (int32_t)sb.members.size());
        }
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            s = KNND_ECUDA;
            break;
        }
        s = make_handle(&sl.h, caps, dtype, precision, prm, sl.stream);
        if (!s) s = balloc(&sl.idx, caps.nK);
        if (!s) s = balloc(&sl.key, caps.nK);
        if (!s) b->ws_bytes += sl.h->ws_bytes + caps.nK * 12;
    }
    for (SubBatch &sb : b->subs) {
        if (s) break;
        s = make_sub_tables(b, sb);
    }
    if (s) {
        batch_free(b);
        return s;
    }
    *out = b;
    return KNND_OK;
}

knnd_status knnd_batch_run(knnd_batch *b, knnd_build_info *info)
{
    if (!b) return KNND_EINVAL;
    // every slot starts after the work already on the caller's stream
    cudaError_t e = cudaEventRecord(b->start, b->stream);
    for (Slot &sl : b->slots)
        if (!e) e = cudaStreamWaitEvent(sl.stream, b->start, 0);
    if (e) return status_of(e);
    // one graph launch per sub-batch; slots take turns so that every stream gets work early
    knnd_status s = KNND_OK;
    size_t most = 0;
    for (const Slot &sl : b->slots) most = std::max(most, sl.subs.size());
    for (size_t k = 0; k < most && !s; ++k) {
        for (Slot &sl : b->slots) {
            if (k >= sl.subs.size()) continue;
            SubBatch &sb = b->subs[sl.subs[k]];
            if (!sb.exec) s = capture_sub(b, sb);
            if (s) break;
            e = cudaGraphLaunch(sb.exec, sl.stream);
            if (e) {
                s = status_of(e);
                break;
            }
        }
    }
    // the caller's stream waits for every slot; the host for everything
    for (Slot &sl : b->slots) {
        cudaEventRecord(sl.done, sl.stream);
        cudaStreamWaitEvent(b->stream, sl.done, 0);
    }
    for (Slot &sl : b->slots) {
        const cudaError_t c = cudaStreamSynchronize(sl.stream);
        if (c && !s) s = status_of(c);
    }
    if (s) return s;
    for (Slot &sl : b->slots) {
        const knnd_status t = take_error(sl.h);
        if (t && !s) s = t;
    }
    if (s) return s;
    const int32_t R = b->prm.max_rounds;
    std::vector<int64_t> upd, hits, resc, fb;
    std::vector<int32_t> rounds, reason;
    for (SubBatch &sb : b->subs) {
        const int32_t ni = (int32_t)sb.members.size();
        rounds.resize(ni);
        e = cudaMemcpy(rounds.data(), sb.hs.rounds, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost);
        if (e) return status_of(e);
        int32_t rmax = 0;
        for (int32_t r : rounds) rmax = std::max(rmax, r);
        b->launches += sb.launches_outer + (int64_t)std::max(0, rmax - 1) * sb.launches_round;
        if (!info) continue;
        upd.resize((size_t)ni * R);
        hits.resize((size_t)ni * (R + 1));
        resc.resize(ni);
        fb.resize(ni);
        reason.resize(ni);
        e = cudaMemcpy(upd.data(), sb.hs.upd, sizeof(int64_t) * ni * R, cudaMemcpyDeviceToHost);
        if (!e) e = cudaMemcpy(hits.data(), sb.hs.hits, sizeof(int64_t) * ni * (R + 1), cudaMemcpyDeviceToHost);
        if (!e) e = cudaMemcpy(resc.data(), sb.hs.rescored, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost);
        if (!e) e = cudaMemcpy(fb.data(), sb.hs.fallback, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost);
        if (!e) e = cudaMemcpy(reason.data(), sb.hs.reason, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost);
        if (e) return status_of(e);
        for (int32_t j = 0; j < ni; ++j) {
            const knnd_instance &in = b->inst[sb.members[j]];
            knnd_build_info &o = info[sb.members[j]];
            std::memset(&o, 0, sizeof(o));
            o.rounds = rounds[j];
            o.stop_reason = reason[j];
            for (int32_t r = 0; r < o.rounds; ++r) o.updates[r] = upd[(size_t)j * R + r];
            for (int32_t r = 0; r <= o.rounds; ++r) o.fcc_hits[r] = hits[(size_t)j * (R + 1) + r];
            o.init_pairs = in.n * in.K;
            o.proposals = (int64_t)o.rounds * in.n * in.K * (2 * (int64_t)in.K + 1);
            o.rescored = resc[j];
            o.merge_fallbacks = fb[j];
            o.join_kernel = sb.join_kernel;
        }
    }
    return KNND_OK;
}

knnd_status knnd_batch_info(const knnd_batch *b, int32_t *sub_batches, int64_t *workspace_bytes,
                            int64_t *kernel_launches)
{
    if (!b) return KNND_EINVAL;
    if (sub_batches) *sub_batches = (int32_t)b->subs.size();
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    if (kernel_launches) *kernel_launches = b->launches;
    return KNND_OK;
}

void knnd_batch_destroy(knnd_batch *b)
{
    if (!b) return;
    for (Slot &sl : b->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

knnd_status knnd_build_batched(int32_t count, const knnd_instance *inst, knnd_dtype dtype, knnd_precision precision,
                               const knnd_params *params, int64_t workspace_limit, knnd_build_info *info,
                               void *stream)
{
    knnd_batch *b = nullptr;
    knnd_status s = knnd_batch_create(&b, count, inst, dtype, precision, params, workspace_limit, stream);
    if (s) return s;
    s = knnd_batch_run(b, info);
    knnd_batch_destroy(b);
    return s;
}

}  // extern "C"
