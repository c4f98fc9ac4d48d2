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
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "knnd_internal.cuh"

using namespace knnd;

namespace {

struct SubBatch {
    int32_t m, K;
    std::vector<int32_t> members;  // indices into the instance array
    int64_t npts;
};

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
    int32_t *nactive;   // 1
};

__global__ void record_hits0_kernel(InstView iv, int32_t ninst, History hs, int32_t max_rounds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    hs.hits[(int64_t)i * (max_rounds + 1)] = iv.cnt[(int64_t)i * kCntNum + kCntHits];
}

// After round r: per-instance stop decision of Sec. 3.3 (iv) (hits of round r
// not above those of round r-1), or no update, or the round cap.
__global__ void stop_kernel(InstView iv, int32_t *active, int32_t ninst, History hs, int32_t r, int32_t max_rounds,
                            int32_t stop_on_zero, float stop_delta, int32_t K)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
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

}  // namespace

struct knnd_batch {
    std::vector<knnd_instance> inst;
    std::vector<SubBatch> subs;
    knnd_dtype dtype;
    knnd_precision prec;
    knnd_params prm;
    cudaStream_t stream;
    knnd_handle *h;   // workspace sized for the largest sub-batch
    int32_t *idx;     // working graph
    double *key;
    const void **ptrs;  // device per-instance tables of the current sub-batch
    int64_t *lds;
    int32_t **oidx;
    double **okey;
    History hs;
    int32_t ninst_cap;
    // pinned host staging
    int64_t *h_base;
    int32_t *h_n;
    uint64_t *h_seed;
    const void **h_ptrs;
    int64_t *h_lds;
    int32_t **h_oidx;
    double **h_okey;
    int32_t *h_nactive;
    int64_t *h_upd, *h_hits, *h_resc, *h_fb;
    int32_t *h_rounds, *h_reason;
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

template <typename T>
knnd_status halloc(T **p, int64_t count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    if (cudaMallocHost((void **)p, sizeof(T) * (size_t)count) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return KNND_ENOMEM;
    }
    return KNND_OK;
}

void batch_free(knnd_batch *b)
{
    if (b->h) destroy_handle(b->h);
    void *dev[] = {b->idx, b->key, b->ptrs, b->lds, b->oidx, b->okey, b->hs.upd, b->hs.hits, b->hs.rescored,
                   b->hs.fallback, b->hs.rounds, b->hs.reason, b->hs.nactive};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *hst[] = {b->h_base, b->h_n, b->h_seed, b->h_ptrs, b->h_lds, b->h_oidx, b->h_okey, b->h_nactive,
                   b->h_upd, b->h_hits, b->h_resc, b->h_fb, b->h_rounds, b->h_reason};
    for (void *p : hst)
        if (p) cudaFreeHost(p);
    delete b;
}

// Device bytes one point of an instance with (m, K) needs in the workspace.
int64_t bytes_per_point(int32_t m, int32_t K, bool mixed, bool incremental)
{
    const int64_t MP = pad_coords(m);
    const int64_t bucket = (int64_t)K * (2 * K + 1) * (mixed ? 8 : 16);
    // tables, per-row scalars, buckets, CSR and arc slots, graph, the split round's graph copy (13 B per arc)
    return MP * 24 + 96 + bucket + (int64_t)K * (4 + 4 + 4 + 8 + 13 + (incremental ? 2 : 0));
}

// One sub-batch: all its instances from points to graphs.
knnd_status run_sub(knnd_batch *b, const SubBatch &sb, knnd_build_info *info)
{
    knnd_handle *h = b->h;
    cudaStream_t st = b->stream;
    const int32_t ni = (int32_t)sb.members.size();
    const int32_t R = b->prm.max_rounds;
    configure(h, sb.npts, sb.m, sb.K);
    h->ninst = ni;
    int64_t off = 0;
    for (int32_t j = 0; j < ni; ++j) {
        const knnd_instance &in = b->inst[sb.members[j]];
        b->h_base[j] = off;
        b->h_n[j] = (int32_t)in.n;
        b->h_seed[j] = in.seed;
        b->h_ptrs[j] = in.points;
        b->h_lds[j] = in.ld;
        b->h_oidx[j] = in.idx;
        b->h_okey[j] = in.key;
        off += in.n;
    }
    b->h_base[ni] = off;
    cudaError_t e = cudaMemcpyAsync(h->inst_base, b->h_base, sizeof(int64_t) * (ni + 1), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(h->inst_n, b->h_n, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(h->inst_seed, b->h_seed, sizeof(uint64_t) * ni, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b->ptrs, b->h_ptrs, sizeof(void *) * ni, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b->lds, b->h_lds, sizeof(int64_t) * ni, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b->oidx, b->h_oidx, sizeof(int32_t *) * ni, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b->okey, b->h_okey, sizeof(double *) * ni, cudaMemcpyHostToDevice, st);
    // every instance active, counters and history cleared
    if (!e) {
        set_ones_kernel<<<(ni + 255) / 256, 256, 0, st>>>(h->inst_active, ni);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemsetAsync(b->hs.rescored, 0, sizeof(int64_t) * ni, st);
    if (!e) e = cudaMemsetAsync(b->hs.fallback, 0, sizeof(int64_t) * ni, st);
    if (!e) e = cudaMemsetAsync(b->hs.upd, 0, sizeof(int64_t) * ni * R, st);
    if (!e) e = cudaMemsetAsync(b->hs.hits, 0, sizeof(int64_t) * ni * (R + 1), st);
    if (e) return status_of(e);
    h->iv.of = h->inst_of;
    h->iv.base = h->inst_base;
    h->iv.n = h->inst_n;
    h->iv.seed = h->inst_seed;
    h->iv.active = h->inst_active;
    h->iv.cnt = h->inst_cnt;
    const int T = 256;
    fill_inst_of_kernel<<<(unsigned)((sb.npts + T - 1) / T), T, 0, st>>>(h->inst_base, ni, sb.npts, h->inst_of);
    h->launches += 1;
    // precompute (EDOMAIN is reported here), initial graphs, clustering hits of G_0
    e = launch_precompute_from(h, nullptr, 0, b->ptrs, b->lds);
    if (e) return status_of(e);
    knnd_status s = take_error(h);
    if (s) return s;
    uint8_t *flag = b->prm.incremental ? h->flag_tmp : nullptr;  // incremental proposals
    e = launch_init_graph(h, 0, b->idx, b->key, flag);
    if (!e) e = cudaMemsetAsync(h->inst_cnt, 0, sizeof(int64_t) * ni * kCntNum, st);
    if (!e) e = launch_fcc_batch(h, b->idx, 0);
    if (e) return status_of(e);
    record_hits0_kernel<<<(ni + T - 1) / T, T, 0, st>>>(h->iv, ni, b->hs, R);
    h->launches += 1;
    for (int32_t r = 1; r <= R; ++r) {
        e = cudaMemsetAsync(h->inst_cnt, 0, sizeof(int64_t) * ni * kCntNum, st);
        if (!e) e = cudaMemsetAsync(b->hs.nactive, 0, sizeof(int32_t), st);
        if (e) return status_of(e);
        s = round_ops(h, 0, r, b->idx, b->key, flag, nullptr);
        if (s) return s;
        e = launch_fcc_batch(h, b->idx, r);
        if (e) return status_of(e);
        stop_kernel<<<(ni + T - 1) / T, T, 0, st>>>(h->iv, h->inst_active, ni, b->hs, r, R,
                                                    b->prm.stop_on_zero_updates, b->prm.stop_delta, sb.K);
        h->launches += 1;
        e = cudaMemcpyAsync(b->h_nactive, b->hs.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) return status_of(e);
        if (*b->h_nactive == 0) break;
    }
    const int64_t nK = sb.npts * sb.K;
    export_kernel<<<(unsigned)((nK + T - 1) / T), T, 0, st>>>(b->idx, b->key, sb.npts, sb.K, h->iv, b->oidx, b->okey);
    h->launches += 1;
    s = take_error(h);
    if (s) return s;
    if (info) {
        e = cudaMemcpyAsync(b->h_upd, b->hs.upd, sizeof(int64_t) * ni * R, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(b->h_hits, b->hs.hits, sizeof(int64_t) * ni * (R + 1), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(b->h_resc, b->hs.rescored, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(b->h_fb, b->hs.fallback, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(b->h_rounds, b->hs.rounds, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(b->h_reason, b->hs.reason, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) return status_of(e);
        for (int32_t j = 0; j < ni; ++j) {
            const knnd_instance &in = b->inst[sb.members[j]];
            knnd_build_info &o = info[sb.members[j]];
            std::memset(&o, 0, sizeof(o));
            o.rounds = b->h_rounds[j];
            o.stop_reason = b->h_reason[j];
            for (int32_t r = 0; r < o.rounds; ++r) o.updates[r] = b->h_upd[(int64_t)j * R + r];
            for (int32_t r = 0; r <= o.rounds; ++r) o.fcc_hits[r] = b->h_hits[(int64_t)j * (R + 1) + r];
            o.init_pairs = in.n * in.K;
            o.proposals = (int64_t)o.rounds * in.n * in.K * (2 * (int64_t)in.K + 1);
            o.rescored = b->h_resc[j];
            o.merge_fallbacks = b->h_fb[j];
        }
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
    if (prm.timing) prm.timing = 0;  // phase timing is a single-instance feature
    const bool mixed = precision != KNND_PREC_FP64;
    for (int32_t i = 0; i < count; ++i) {
        const knnd_instance &in = inst[i];
        if (!in.points || !in.idx || !in.key) return KNND_EINVAL;
        if (in.n < 3 || in.n >= ((int64_t)1 << 31)) return KNND_EINVAL;
        if (in.m < 1 || in.m > KNND_MAX_M || in.ld < in.m) return KNND_EINVAL;
        if (in.K < 2 || in.K > KNND_MAX_K || (int64_t)in.K >= in.n) return KNND_EINVAL;
    }
    if (workspace_limit <= 0) workspace_limit = (int64_t)32 << 30;
    // classes by (m, K); sub-batches within the budget, in input order
    std::map<std::pair<int32_t, int32_t>, std::vector<int32_t>> classes;
    for (int32_t i = 0; i < count; ++i) classes[{inst[i].m, inst[i].K}].push_back(i);
    knnd_batch *b = new (std::nothrow) knnd_batch();
    if (!b) return KNND_ENOMEM;
    b->inst.assign(inst, inst + count);
    b->dtype = dtype;
    b->prec = precision;
    b->prm = prm;
    b->stream = (cudaStream_t)stream;
    Caps caps = {0, 0, 0, 0, 0};
    for (auto &kv : classes) {
        const int32_t m = kv.first.first, K = kv.first.second;
        const int64_t bpp = bytes_per_point(m, K, mixed, prm.incremental != 0);
        SubBatch cur{m, K, {}, 0};
        auto flush = [&]() {
            if (cur.members.empty()) return;
            caps.n = std::max(caps.n, cur.npts);
            caps.tab = std::max(caps.tab, cur.npts * pad_coords(m));
            caps.nK = std::max(caps.nK, cur.npts * K);
            caps.bucket = std::max(caps.bucket, cur.npts * K * (2 * (int64_t)K + 1));
            caps.ninst = std::max(caps.ninst, (int32_t)cur.members.size());
            b->subs.push_back(cur);
            cur = SubBatch{m, K, {}, 0};
        };
        for (int32_t i : kv.second) {
            const int64_t ni = inst[i].n;
            const bool over = (cur.npts + ni) * bpp > workspace_limit ||
                              (int64_t)K * K + (int64_t)(K + 1) * (cur.npts + ni) >= ((int64_t)1 << 31);
            if (!cur.members.empty() && over) flush();
            cur.members.push_back(i);
            cur.npts += ni;
        }
        flush();
    }
    const int32_t R = prm.max_rounds, ni = caps.ninst;
    b->ninst_cap = ni;
    knnd_status s = make_handle(&b->h, caps, dtype, precision, prm, stream);
    if (!s) s = balloc(&b->idx, caps.nK);
    if (!s) s = balloc(&b->key, caps.nK);
    if (!s) s = balloc(&b->ptrs, ni);
    if (!s) s = balloc(&b->lds, ni);
    if (!s) s = balloc(&b->oidx, ni);
    if (!s) s = balloc(&b->okey, ni);
    if (!s) s = balloc(&b->hs.upd, (int64_t)ni * R);
    if (!s) s = balloc(&b->hs.hits, (int64_t)ni * (R + 1));
    if (!s) s = balloc(&b->hs.rescored, ni);
    if (!s) s = balloc(&b->hs.fallback, ni);
    if (!s) s = balloc(&b->hs.rounds, ni);
    if (!s) s = balloc(&b->hs.reason, ni);
    if (!s) s = balloc(&b->hs.nactive, 1);
    if (!s) s = halloc(&b->h_base, ni + 1);
    if (!s) s = halloc(&b->h_n, ni);
    if (!s) s = halloc(&b->h_seed, ni);
    if (!s) s = halloc(&b->h_ptrs, ni);
    if (!s) s = halloc(&b->h_lds, ni);
    if (!s) s = halloc(&b->h_oidx, ni);
    if (!s) s = halloc(&b->h_okey, ni);
    if (!s) s = halloc(&b->h_nactive, 1);
    if (!s) s = halloc(&b->h_upd, (int64_t)ni * R);
    if (!s) s = halloc(&b->h_hits, (int64_t)ni * (R + 1));
    if (!s) s = halloc(&b->h_resc, ni);
    if (!s) s = halloc(&b->h_fb, ni);
    if (!s) s = halloc(&b->h_rounds, ni);
    if (!s) s = halloc(&b->h_reason, ni);
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
    for (const SubBatch &sb : b->subs) {
        knnd_status s = run_sub(b, sb, info);
        if (s) return s;
    }
    return KNND_OK;
}

knnd_status knnd_batch_info(const knnd_batch *b, int32_t *sub_batches, int64_t *workspace_bytes,
                            int64_t *kernel_launches)
{
    if (!b) return KNND_EINVAL;
    if (sub_batches) *sub_batches = (int32_t)b->subs.size();
    if (workspace_bytes) *workspace_bytes = b->h ? b->h->ws_bytes : 0;
    if (kernel_launches) *kernel_launches = b->h ? b->h->launches : 0;
    return KNND_OK;
}

void knnd_batch_destroy(knnd_batch *b)
{
    if (!b) return;
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
