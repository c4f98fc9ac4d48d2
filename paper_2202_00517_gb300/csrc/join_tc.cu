// join_tc.cu -- the join tile on the 5th-generation tensor cores (tcgen05),
// BF16 hi/lo split products with FP32 accumulation in tensor memory.
//
// The hub tile of Sec. 3.1 (rows F(v) + coF(v), columns F(v) and v) is the
// contraction D[r][c] = <x_r, log y_c>.  Each FP32 operand is split into two
// BF16 terms, a = a_hi + a_lo; the tile is a_hi b_hi + a_hi b_lo + a_lo b_hi,
// three tcgen05.mma per 16-wide k step, accumulated in FP32 in TMEM.
// |D~ - <x, log y>| <= c_tc sum_i |x_i log y_i| with
//   c_tc = 3 * 2^-16           (dropped a_lo b_lo and the split residuals)
//        + 2^-24               (log y rounded to FP32)
//        + (3 KD + 8) 2^-22    (FP32 accumulation, not assumed round-to-nearest)
// times 1.05; the filter and the FP64 re-score of the merge use that bound
// exactly as for the CUDA-core FP32 form, so the graph is the FP64 form's.
//
// One CTA of four warps takes one hub at a time.  The columns (K of F(v) and
// v itself, padded to N = a multiple of 16) and up to 128 rows are converted
// into shared memory in the K-major canonical layout without swizzle (8 x 8
// core matrices of 128 contiguous bytes; 128 B between core matrices along K,
// KD / 8 * 128 B between 8-row groups).  Thread 0 issues the MMAs into a
// 128 x N FP32 accumulator in TMEM and commits them to an mbarrier; every
// thread then reads its own row (TMEM lane) with tcgen05.ld, applies the
// filter and compacts its survivors, and the warp writes them coalesced.
// Every wait is bounded (1 s of the global timer); a timeout sets kErrTimeout,
// waits (bounded) for MMAs it issued, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "knnd_internal.cuh"

namespace knnd {

struct TcArgs {
    int64_t n;
    int64_t h_lo, h_hi;  // the hubs this launch takes: [h_lo, h_hi), those of phase `phase` (in_phase)
    int phase, split_den;
    int K;
    const int32_t *idx;
    const int64_t *cof_off;
    const int32_t *cof;
    const float *X32;
    const float *L32;
    const RowMeta *meta;
    int32_t *bcnt;
    int2 *bent;
    int32_t *err;
    int debug;
    InstView iv;
    // incremental proposals (as in join.cu): flags of G_{r-1} and of the coF
    // entries, or NULL
    const uint8_t *flag;
    const uint8_t *cof_new;
    // bound audit (debug)
    const double *X64;
    const double *L64;
    const double *negH;
    const double *Ex;
    int64_t *cnt;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, K-direction core-matrix stride (lbo),
// 8-row-group stride (sbo), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

template <int KD, int N>
struct TcLayout {
    static constexpr int M = 128;
    static constexpr int SBO_A = KD / 8 * 128;
    static constexpr int SBO_B = KD / 8 * 128;
    static constexpr int A_BYTES = M * KD * 2;  // one of hi / lo
    static constexpr int B_BYTES = N * KD * 2;
    static constexpr int DS = N | 1;            // odd row stride of the dots (floats)
    static constexpr int JS = (N + 3) & ~3;     // row stride of the survivor columns (bytes)
    static constexpr int W_SCRATCH = 32 * DS * 4 + 32 * JS + 32 * 4 + 32 * 8;
    static constexpr int A_REGION = (2 * A_BYTES > 4 * W_SCRATCH) ? 2 * A_BYTES : ((4 * W_SCRATCH + 127) & ~127);
    static constexpr int OFF_AH = 0;
    static constexpr int OFF_AL = A_BYTES;
    static constexpr int OFF_BH = A_REGION;
    static constexpr int OFF_BL = OFF_BH + B_BYTES;
    static constexpr int OFF_CID = OFF_BL + B_BYTES;
    static constexpr int OFF_CNEW = OFF_CID + ((N * 4 + 127) & ~127);  // new-flags of the columns
    static constexpr int OFF_MISC = OFF_CNEW + ((N + 127) & ~127);
    static constexpr int BYTES = OFF_MISC + 128;
    static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
};

__device__ __forceinline__ void split_store(const float4 a, const float4 b, __nv_bfloat16 *hi, __nv_bfloat16 *lo)
{
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        h[i] = __float2bfloat16_rn(v[i]);
        l[i] = __float2bfloat16_rn(v[i] - __bfloat162float(h[i]));
    }
    *reinterpret_cast<uint4 *>(hi) = *reinterpret_cast<const uint4 *>(h);
    *reinterpret_cast<uint4 *>(lo) = *reinterpret_cast<const uint4 *>(l);
}

constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Polls the mbarrier phase `parity` until it completes (true) or `limit` ns pass (false).
__device__ __forceinline__ bool mbar_wait_ns(uint32_t bar, uint32_t parity, unsigned long long limit)
{
    const unsigned long long t0 = global_ns();
    for (int it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63) == 63 && global_ns() - t0 > limit) return false;
    }
}

// 64 registers (eight CTAs per SM) while the accumulator row is at most 32 wide;
// wider rows keep theirs in registers at 128
template <int MP, int KD, int N>
__global__ void __launch_bounds__(128, N <= 32 ? 8 : 4) join_tc_kernel(TcArgs a)
{
    using Lay = TcLayout<KD, N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sAh = smem + Lay::OFF_AH;
    unsigned char *sAl = smem + Lay::OFF_AL;
    unsigned char *sBh = smem + Lay::OFF_BH;
    unsigned char *sBl = smem + Lay::OFF_BL;
    int *sCid = reinterpret_cast<int *>(smem + Lay::OFF_CID);
    unsigned char *sCnew = smem + Lay::OFF_CNEW;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smem + Lay::OFF_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + Lay::OFF_MISC + 8);
    int *sAbort = reinterpret_cast<int *>(smem + Lay::OFF_MISC + 16);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int K = a.K;
    const int64_t n = a.n;
    const unsigned FULL = 0xffffffffu;

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sAbort = 0;
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)Lay::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *tslot;
    uint32_t phase = 0;
    bool first_tile = true;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                           ((uint32_t)(Lay::M >> 4) << 24);
    // per-warp epilogue scratch, aliased on the A operands once the MMAs completed
    unsigned char *wsc = smem + w * Lay::W_SCRATCH;
    float *sD = reinterpret_cast<float *>(wsc);
    unsigned char *sJ = wsc + 32 * Lay::DS * 4;
    int *sInc = reinterpret_cast<int *>(sJ + 32 * Lay::JS);
    int64_t *sRB = reinterpret_cast<int64_t *>(sInc + 32);
    int64_t ndot = 0, nviol = 0;

    for (int64_t v = a.h_lo + blockIdx.x; v < a.h_hi; v += gridDim.x) {
        if (!a.iv.live(v)) continue;
        if (!in_phase(a.iv, a.phase, a.split_den, n, v)) continue;
        if (a.flag) {  // incremental proposals: a hub with no new arc has nothing to propose
            const int64_t h0 = a.cof_off[v], hn = (int64_t)K + (a.cof_off[v + 1] - h0);
            int any = 0;
            for (int64_t r = t; r < hn; r += blockDim.x)
                any |= (r < K ? a.flag[v * K + r] : a.cof_new[h0 + (r - K)]) != 0;
            if (!__syncthreads_or(any)) continue;
        }
        // columns: F(v), then v itself (the co-friend column of the rows of F(v))
        for (int j = t; j < N; j += blockDim.x) {
            int id = -1;
            int nw = 0;
            if (j < K) {
                id = a.idx[v * K + j];
                nw = a.flag ? a.flag[v * K + j] : 1;
                if (id < 0 || id >= n) {
                    atomicOr(a.err, kErrIndex);
                    id = -1;
                }
            } else if (j == K) {
                id = (int)v;
            }
            sCid[j] = id;
            sCnew[j] = (unsigned char)nw;
        }
        __syncthreads();
        for (int u = t; u < N * (KD / 8); u += blockDim.x) {
            const int j = u / (KD / 8), c8 = u - j * (KD / 8);
            const int id = sCid[j];
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = p;
            if (id >= 0 && 8 * c8 < MP) {
                const float4 *src = reinterpret_cast<const float4 *>(a.L32 + (int64_t)id * MP + 8 * c8);
                p = __ldg(src);
                q = __ldg(src + 1);
            }
            const int off = (j >> 3) * Lay::SBO_B + c8 * 128 + (j & 7) * 16;
            split_store(p, q, reinterpret_cast<__nv_bfloat16 *>(sBh + off),
                        reinterpret_cast<__nv_bfloat16 *>(sBl + off));
        }
        const int64_t c0 = a.cof_off[v];
        const int64_t nrows = (int64_t)K + (a.cof_off[v + 1] - c0);
        for (int64_t base = 0; base < nrows; base += Lay::M) {
            // rows: thread t <-> row base + t
            const int64_t r = base + t;
            int rid = -1, rnew = 1;
            if (r < nrows) {
                rid = (r < K) ? a.idx[v * K + r] : a.cof[c0 + (r - K)];
                if (a.flag) rnew = (r < K) ? a.flag[v * K + r] : a.cof_new[c0 + (r - K)];
                if (rid < 0 || rid >= n) {
                    atomicOr(a.err, kErrIndex);
                    rid = -1;
                }
            }
            float ph = 0.f;
            int64_t boff = 0;
            if (rid >= 0) {
                const RowMeta rm = a.meta[rid];
                ph = rm.phi;
                boff = rm.boff;
            }
#pragma unroll
            for (int c8 = 0; c8 < KD / 8; ++c8) {
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = p;
                if (rid >= 0 && 8 * c8 < MP) {
                    const float4 *src = reinterpret_cast<const float4 *>(a.X32 + (int64_t)rid * MP + 8 * c8);
                    p = __ldg(src);
                    q = __ldg(src + 1);
                }
                const int off = (t >> 3) * Lay::SBO_A + c8 * 128 + (t & 7) * 16;
                split_store(p, q, reinterpret_cast<__nv_bfloat16 *>(sAh + off),
                            reinterpret_cast<__nv_bfloat16 *>(sAl + off));
            }
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            // debug == 2: block 0's first tile issues nothing, so its wait below runs
            // out (the bounded-wait path, tested without a fault)
            const bool issue = !(a.debug == 2 && blockIdx.x == 0 && first_tile);
            first_tile = false;
            if (t == 0 && issue) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
                for (int s = 0; s < KD / 16; ++s) {
                    const uint64_t dah = umma_desc(ah + s * 256, 128, Lay::SBO_A);
                    const uint64_t dal = umma_desc(al + s * 256, 128, Lay::SBO_A);
                    const uint64_t dbh = umma_desc(bh + s * 256, 128, Lay::SBO_B);
                    const uint64_t dbl = umma_desc(bl + s * 256, 128, Lay::SBO_B);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                                 "l"(dah), "l"(dbh), "r"(idesc), "r"(acc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(taddr), "l"(dah),
                                 "l"(dbl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(taddr), "l"(dal),
                                 "l"(dbh), "r"(idesc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(mbar)));
            }
            // bounded wait for the MMAs (1 s of the global timer)
            bool done = mbar_wait_ns(smem_u32(mbar), phase, kWaitNs);
            if (!done) {
                atomicOr(a.err, kErrTimeout);
                atomicOr(sAbort, 1);
                // MMAs that were issued may still be writing the accumulator: give
                // them a second bounded wait before the TMEM is freed
                if (issue) mbar_wait_ns(smem_u32(mbar), phase, kWaitNs);
            }
            phase ^= 1u;
            __syncthreads();
            if (*sAbort) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // this thread's row of the accumulator -> its row of the warp scratch
            // (the scratch aliases the A operands, free once every warp is here)
            uint32_t u[N];
#pragma unroll
            for (int c = 0; c < N; c += 16) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(u[c + 0]), "=r"(u[c + 1]), "=r"(u[c + 2]), "=r"(u[c + 3]), "=r"(u[c + 4]),
                               "=r"(u[c + 5]), "=r"(u[c + 6]), "=r"(u[c + 7]), "=r"(u[c + 8]), "=r"(u[c + 9]),
                               "=r"(u[c + 10]), "=r"(u[c + 11]), "=r"(u[c + 12]), "=r"(u[c + 13]), "=r"(u[c + 14]),
                               "=r"(u[c + 15])
                             : "r"(taddr + ((uint32_t)(32 * w) << 16) + (uint32_t)c));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            float *drow = sD + lane * Lay::DS;
#pragma unroll
            for (int j = 0; j < N; ++j) drow[j] = __uint_as_float(u[j]);
            // filter, compacting the survivors in place; the co-friend column v
            // (index K) counts for rows of F(v) only
            int q = 0;
            if (rid >= 0) {
                for (int j = 0; j <= K; ++j) {
                    const int cj = sCid[j];
                    if (cj < 0 || cj == rid || (j == K && r >= K)) continue;
                    const float dj = drow[j];
                    if (a.debug) {  // bound audit: |D~ - FP64 dot| <= E_x
                        const double *xr = a.X64 + (int64_t)rid * MP;
                        const double *lr = a.L64 + (int64_t)cj * MP;
                        double acc = 0.0;
                        for (int i = 0; i < MP; ++i) acc = __fma_rn(xr[i], lr[i], acc);
                        ndot += 1;
                        if (fabs((double)dj - acc) > a.Ex[rid]) nviol += 1;
                    }
                    // incremental: a pair met only through arcs of G_{r-2} is not proposed again
                    if (dj >= ph && (rnew || sCnew[j])) {
                        drow[q] = dj;
                        sJ[lane * Lay::JS + q] = (unsigned char)j;
                        ++q;
                    }
                }
            }
            int64_t rowbase = -1;
            if (q > 0) {
                const int p = atomicAdd(&a.bcnt[rid], q);
                rowbase = boff + p;
                if (a.debug) {
                    const int64_t cap = (int64_t)K * K + (int64_t)(K + 1) * (a.cof_off[rid + 1] - a.cof_off[rid]);
                    if (p + q > cap) {
                        atomicOr(a.err, kErrBucket);
                        rowbase = -1;
                    }
                }
            }
            // coalesced writes of the warp's survivors (flattened over its 32 rows)
            int incl = q;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tt = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += tt;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            sInc[lane] = incl;
            sRB[lane] = rowbase;
            __syncwarp();
            for (int k = lane; k < total; k += 32) {
                int lo = 0, hi = 31;
#pragma unroll
                for (int it = 0; it < 5; ++it) {
                    const int mid = (lo + hi) >> 1;
                    if (sInc[mid] > k) hi = mid;
                    else lo = mid + 1;
                }
                const int qq = k - (lo ? sInc[lo - 1] : 0);
                const int64_t rb = sRB[lo];
                if (rb >= 0)
                    a.bent[rb + qq] = make_int2((int)sortable_bits(-sD[lo * Lay::DS + qq]), sCid[sJ[lo * Lay::JS + qq]]);
            }
            __syncthreads();  // scratch free before the next tile's operands
        }
        if (*sAbort) break;
        __syncthreads();  // columns free before the next hub
    }
    if (a.debug && (ndot || nviol)) {
        atomicAdd((unsigned long long *)&a.cnt[kCntBoundViol], (unsigned long long)nviol);
        atomicAdd((unsigned long long *)&a.cnt[kCntAudited], (unsigned long long)ndot);
    }
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                             "r"((uint32_t)Lay::TMEM_COLS));
}

// Resident CTAs per SM from the device's limits: shared memory (with the
// per-block reservation), registers, threads, and TMEM (512 columns per SM,
// each CTA holding `tmem_cols` for its lifetime).  The runtime's occupancy
// query answers 1 for this kernel, which left the GPU with one hub in flight
// per SM.
static int tc_blocks_per_sm(const void *fn, size_t smem, int threads, int tmem_cols, int device)
{
    int smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, device);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp, 256 at a time
    int n = 512 / tmem_cols;
    n = std::min(n, smem_sm / (int)(smem + resv));
    n = std::min(n, regs_sm / (regs_warp * (threads / 32)));
    n = std::min(n, thr_sm / threads);
    return std::max(n, 1);
}

template <int MP, int KD, int N>
static cudaError_t run_tc(knnd_handle *h, const TcArgs &a)
{
    using Lay = TcLayout<KD, N>;
    const int threads = 128;
    const size_t smem = Lay::BYTES;
    cudaFuncSetAttribute(join_tc_kernel<MP, KD, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(join_tc_kernel<MP, KD, N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    const int per_sm =
        tc_blocks_per_sm((const void *)join_tc_kernel<MP, KD, N>, smem, threads, Lay::TMEM_COLS, h->device);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.h_hi - a.h_lo, (int64_t)h->num_sms * per_sm));
    join_tc_kernel<MP, KD, N><<<(unsigned)grid, threads, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <int MP, int KD>
static cudaError_t run_tc_n(knnd_handle *h, const TcArgs &a)
{
    const int need = h->K + 1;  // F(v) and v
    if (need <= 16) return run_tc<MP, KD, 16>(h, a);
    if (need <= 32) return run_tc<MP, KD, 32>(h, a);
    if (need <= 48) return run_tc<MP, KD, 48>(h, a);
    if (need <= 64) return run_tc<MP, KD, 64>(h, a);
    return run_tc<MP, KD, 80>(h, a);
}

bool tc_supported(int MP, int K) { return MP >= 8 && MP <= 128 && K + 1 <= 80; }

cudaError_t launch_join_tc(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase,
                           int split_den)
{
    TcArgs a;
    a.n = h->n;
    a.h_lo = h_lo;
    a.h_hi = h_hi;
    a.phase = phase;
    a.split_den = split_den;
    a.K = h->K;
    a.idx = idx;
    a.cof_off = h->cof_off;
    a.cof = h->cof;
    a.X32 = h->X32;
    a.L32 = h->L32;
    a.meta = h->meta;
    a.bcnt = h->bcnt;
    a.bent = h->bent;
    a.err = h->err;
    a.debug = h->prm.debug;
    a.iv = h->iv;
    a.flag = h->round_flag;
    a.cof_new = h->round_flag ? h->cof_new : nullptr;
    a.X64 = h->X64;
    a.L64 = h->L64;
    a.negH = h->negH;
    a.Ex = h->Ex;
    a.cnt = h->cnt;
    cudaMemsetAsync(h->bcnt, 0, sizeof(int32_t) * h->n, h->stream);
    h->launches += 1;
    switch (h->MP) {
    case 8: return run_tc_n<8, 16>(h, a);
    case 16: return run_tc_n<16, 16>(h, a);
    case 24: return run_tc_n<24, 32>(h, a);
    case 32: return run_tc_n<32, 32>(h, a);
    case 48: return run_tc_n<48, 48>(h, a);
    case 64: return run_tc_n<64, 64>(h, a);
    case 72: return run_tc_n<72, 80>(h, a);
    case 96: return run_tc_n<96, 96>(h, a);
    case 128: return run_tc_n<128, 128>(h, a);
    default: return cudaErrorInvalidValue;
    }
}

// c_tc of the BF16 x 3 tile (see the file header), for KD = m padded to 16.
double bound_c_bf16x3(int MP)
{
    const int KD = (MP + 15) / 16 * 16;
    return (3.0 * 0x1p-16 + 0x1p-24 + (3.0 * KD + 8.0) * 0x1p-22) * 1.05;
}

}  // namespace knnd
