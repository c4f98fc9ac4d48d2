// merge.cu -- the bounded top-K update of one round (Sec. 3.1 "Update",
// Sec. 4.2 NavigableSet insertion): the new friend list of x is the K best,
// under (key ascending, index ascending), of its old list and the candidates
// the join appended to its bucket; duplicates and x itself never enter.
//
// One warp per point x.  The list lives in registers, entry q = lane + 32*e
// (e < NE, NE = 1 for K <= 32, 2 for K <= 64).  A candidate that beats the
// K-th entry is inserted by one ballot (rank), one shuffle-up (shift) and a
// select; a ballot of index equality rejects duplicates.
//
// FP64 form: bucket entries carry exact keys.
// Mixed form: bucket entries carry the FP32 dot d~; the exact key lies in
// [negH - d~ - E_x, negH - d~ + E_x].  Pass A keeps the K best upper bounds
// (old entries: exact keys) -> T, an upper bound of the exact K-th key of the
// whole pool.  Pass B re-scores in FP64 (canonical fma chain) only the
// candidates whose lower bound is <= T and <= the current exact K-th key and
// that are not already in the exact list, and inserts them.  The result equals
// the FP64 form's bit for bit.
#include <algorithm>

#include "knnd_internal.cuh"

namespace knnd {

template <int NE>
struct WarpList {
    double k[NE];
    int i[NE];
    int old[NE];

    __device__ __forceinline__ void kth(int K, double &kk, int &ik) const {
        const int e = (K - 1) >> 5, src = (K - 1) & 31;
        double kv = k[0];
        int iv = i[0];
#pragma unroll
        for (int t = 1; t < NE; ++t)
            if (e == t) {
                kv = k[t];
                iv = i[t];
            }
        kk = __shfl_sync(0xffffffffu, kv, src);
        ik = __shfl_sync(0xffffffffu, iv, src);
    }
    __device__ __forceinline__ bool contains(int K, int lane, int y) const {
        bool f = false;
#pragma unroll
        for (int e = 0; e < NE; ++e) f |= (lane + 32 * e < K) && (i[e] == y);
        return __any_sync(0xffffffffu, f);
    }
    // insert (ck, ci) which is known to be better than the K-th entry and absent
    __device__ __forceinline__ void insert(int K, int lane, double ck, int ci, int cold) {
        int p = 0;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const bool less = (lane + 32 * e < K) && lex_less(k[e], i[e], ck, ci);
            p += __popc(__ballot_sync(0xffffffffu, less));
        }
        double uk[NE];
        int ui[NE], uo[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            uk[e] = __shfl_up_sync(0xffffffffu, k[e], 1);
            ui[e] = __shfl_up_sync(0xffffffffu, i[e], 1);
            uo[e] = __shfl_up_sync(0xffffffffu, old[e], 1);
        }
#pragma unroll
        for (int e = NE - 1; e >= 0; --e) {
            if (e > 0) {  // lane 0 of slot e takes lane 31 of slot e-1
                const double ck2 = __shfl_sync(0xffffffffu, k[e - 1], 31);
                const int ci2 = __shfl_sync(0xffffffffu, i[e - 1], 31);
                const int co2 = __shfl_sync(0xffffffffu, old[e - 1], 31);
                if (lane == 0) {
                    uk[e] = ck2;
                    ui[e] = ci2;
                    uo[e] = co2;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int q = lane + 32 * e;
            if (q == p) {
                k[e] = ck;
                i[e] = ci;
                old[e] = cold;
            } else if (q > p) {
                k[e] = uk[e];
                i[e] = ui[e];
                old[e] = uo[e];
            }
        }
    }
};

struct MergeArgs {
    int64_t n;
    int K;
    int MP;
    int32_t *idx;
    double *key;
    uint8_t *flag;
    const int64_t *cof_off;
    const int32_t *bcnt;
    const int2 *bent;
    const double *bkey;
    const int32_t *bidx;
    const double *X64;
    const double *L64;
    const double *negH;
    const double *Ex;
    int64_t *cnt;
    int32_t *err;
};

template <int NE>
__device__ __forceinline__ void write_row(const MergeArgs &a, int64_t x, int lane, const WarpList<NE> &X,
                                          int &newcount)
{
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int q = lane + 32 * e;
        if (q < a.K) {
            a.idx[x * a.K + q] = X.i[e];
            a.key[x * a.K + q] = X.k[e];
            if (a.flag) a.flag[x * a.K + q] = X.old[e] ? 0 : 1;
            newcount += X.old[e] ? 0 : 1;
        }
    }
}

template <int NE>
__device__ __forceinline__ void load_row(const MergeArgs &a, int64_t x, int lane, WarpList<NE> &X)
{
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int q = lane + 32 * e;
        if (q < a.K) {
            X.k[e] = a.key[x * a.K + q];
            X.i[e] = a.idx[x * a.K + q];
        } else {
            X.k[e] = 0.0;
            X.i[e] = -1;
        }
        X.old[e] = 1;
    }
}

// Lane-parallel test of y against the row's original list (indices `oi`, entry
// q = lane + 32 e): every lane checks its own candidate, K shuffles in all.
template <int NE>
__device__ __forceinline__ bool in_old_list(const int (&oi)[NE], int K, int y)
{
    bool f = false;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int lim = min(32, K - 32 * e);
        for (int t = 0; t < lim; ++t) f |= (__shfl_sync(0xffffffffu, oi[e], t) == y);
    }
    return f;
}

// Entries the join wrote for x, never more than the row's capacity.
__device__ __forceinline__ int bucket_count(const MergeArgs &a, int64_t x)
{
    const int64_t cap = (int64_t)a.K * a.K + (int64_t)(a.K + 1) * (a.cof_off[x + 1] - a.cof_off[x]);
    const int c = a.bcnt[x];
    if (c > cap) {
        if ((threadIdx.x & 31) == 0) atomicOr(a.err, kErrBucket);
        return (int)cap;
    }
    return c;
}

__device__ __forceinline__ void flush_updates(int64_t *cnt, int newcount)
{
    for (int o = 16; o > 0; o >>= 1) newcount += __shfl_xor_sync(0xffffffffu, newcount, o);
    if ((threadIdx.x & 31) == 0 && newcount) atomicAdd((unsigned long long *)&cnt[kCntUpdates], (unsigned long long)newcount);
}

// ------------------------------------------------------------------ FP64 form
template <int NE>
__global__ void __launch_bounds__(256) merge_fp64_kernel(MergeArgs a)
{
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int K = a.K;
    int newcount = 0;
    for (int64_t x = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); x < a.n; x += (int64_t)gridDim.x * wpb) {
        WarpList<NE> X;
        load_row(a, x, lane, X);
        int oi[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) oi[e] = X.i[e];
        double tk;
        int ti;
        X.kth(K, tk, ti);
        const int64_t base = (int64_t)K * K * x + (int64_t)(K + 1) * a.cof_off[x];
        const int cnt = bucket_count(a, x);
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const bool has = c0 + lane < cnt;
            double ck = 0.0;
            int ci = -1;
            if (has) {
                ck = a.bkey[base + c0 + lane];
                ci = a.bidx[base + c0 + lane];
            }
            const bool old = in_old_list(oi, K, ci);
            unsigned mask = __ballot_sync(0xffffffffu, has && !old && lex_less(ck, ci, tk, ti));
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const double k1 = __shfl_sync(0xffffffffu, ck, src);
                const int i1 = __shfl_sync(0xffffffffu, ci, src);
                if (!lex_less(k1, i1, tk, ti)) continue;
                if (X.contains(K, lane, i1)) continue;
                X.insert(K, lane, k1, i1, 0);
                X.kth(K, tk, ti);
            }
        }
        write_row(a, x, lane, X, newcount);
    }
    flush_updates(a.cnt, newcount);
}

// ------------------------------------------------------------------ mixed form
template <int NE>
__global__ void __launch_bounds__(256) merge_mixed_kernel(MergeArgs a)
{
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int K = a.K;
    const int MP = a.MP;
    int newcount = 0;
    long long rescored = 0;
    for (int64_t x = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); x < a.n; x += (int64_t)gridDim.x * wpb) {
        WarpList<NE> X;
        load_row(a, x, lane, X);
        int oi[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) oi[e] = X.i[e];
        const int64_t base = (int64_t)K * K * x + (int64_t)(K + 1) * a.cof_off[x];
        const int cnt = bucket_count(a, x);
        if (cnt > 0) {
            const double nh = a.negH[x];
            const double E = a.Ex[x];
            // pass A: K best upper bounds
            WarpList<NE> A = X;
            double tk, xk;
            int ti, xi;
            A.kth(K, tk, ti);
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const bool has = c0 + lane < cnt;
                double ub = 0.0;
                int ci = -1;
                if (has) {
                    const int2 en = a.bent[base + c0 + lane];
                    ub = (nh - (double)__int_as_float(en.x)) + E;
                    ci = en.y;
                }
                // old friends re-proposed by the join are dropped without serial work
                const bool old = in_old_list(oi, K, ci);
                unsigned mask = __ballot_sync(0xffffffffu, has && !old && lex_less(ub, ci, tk, ti));
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const double k1 = __shfl_sync(0xffffffffu, ub, src);
                    const int i1 = __shfl_sync(0xffffffffu, ci, src);
                    if (!lex_less(k1, i1, tk, ti)) continue;
                    if (A.contains(K, lane, i1)) continue;
                    A.insert(K, lane, k1, i1, 0);
                    A.kth(K, tk, ti);
                }
            }
            const double T = tk;
            // pass B: exact re-score of the candidates the bounds cannot reject
            X.kth(K, xk, xi);
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const bool has = c0 + lane < cnt;
                double lb = 0.0;
                int ci = -1;
                if (has) {
                    const int2 en = a.bent[base + c0 + lane];
                    lb = (nh - (double)__int_as_float(en.x)) - E;
                    ci = en.y;
                }
                const bool old = in_old_list(oi, K, ci);  // warp-collective: every lane calls it
                bool want = has && !old && lb <= T && lb <= xk && ci >= 0 && ci < a.n;
                unsigned mask = __ballot_sync(0xffffffffu, want);
                // drop candidates already in the exact list
                unsigned m2 = mask;
                while (m2) {
                    const int src = __ffs(m2) - 1;
                    m2 &= m2 - 1;
                    const int i1 = __shfl_sync(0xffffffffu, ci, src);
                    if (X.contains(K, lane, i1) && lane == src) want = false;
                }
                double kex = 0.0;
                if (want) {
                    const double2 *xr = reinterpret_cast<const double2 *>(a.X64 + x * MP);
                    const double2 *lr = reinterpret_cast<const double2 *>(a.L64 + (int64_t)ci * MP);
                    double acc = 0.0;
                    for (int i2 = 0; i2 < MP / 2; ++i2) {
                        const double2 p = __ldg(xr + i2), q = __ldg(lr + i2);
                        acc = __fma_rn(p.x, q.x, acc);
                        acc = __fma_rn(p.y, q.y, acc);
                    }
                    kex = nh - acc;
                    rescored += 1;
                }
                mask = __ballot_sync(0xffffffffu, want);
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const double k1 = __shfl_sync(0xffffffffu, kex, src);
                    const int i1 = __shfl_sync(0xffffffffu, ci, src);
                    if (!lex_less(k1, i1, xk, xi)) continue;
                    if (X.contains(K, lane, i1)) continue;
                    X.insert(K, lane, k1, i1, 0);
                    X.kth(K, xk, xi);
                }
            }
        }
        write_row(a, x, lane, X, newcount);
    }
    flush_updates(a.cnt, newcount);
    for (int o = 16; o > 0; o >>= 1) rescored += __shfl_xor_sync(0xffffffffu, rescored, o);
    if (lane == 0 && rescored) atomicAdd((unsigned long long *)&a.cnt[kCntRescored], (unsigned long long)rescored);
}

cudaError_t launch_merge(knnd_handle *h, int32_t *idx, double *key, uint8_t *newflag)
{
    MergeArgs a;
    a.n = h->n;
    a.K = h->K;
    a.MP = h->MP;
    a.idx = idx;
    a.key = key;
    a.flag = newflag;
    a.cof_off = h->cof_off;
    a.bcnt = h->bcnt;
    a.bent = h->bent;
    a.bkey = h->bkey;
    a.bidx = h->bidx;
    a.X64 = h->X64;
    a.L64 = h->L64;
    a.negH = h->negH;
    a.Ex = h->Ex;
    a.cnt = h->cnt;
    a.err = h->err;
    const int threads = 256;
    const int64_t need = (h->n + threads / 32 - 1) / (threads / 32);
    const int64_t grid = std::min<int64_t>(need, (int64_t)h->num_sms * 8);
    const bool fp64 = h->prec == KNND_PREC_FP64;
    if (h->K <= 32) {
        if (fp64) merge_fp64_kernel<1><<<(unsigned)grid, threads, 0, h->stream>>>(a);
        else merge_mixed_kernel<1><<<(unsigned)grid, threads, 0, h->stream>>>(a);
    } else {
        if (fp64) merge_fp64_kernel<2><<<(unsigned)grid, threads, 0, h->stream>>>(a);
        else merge_mixed_kernel<2><<<(unsigned)grid, threads, 0, h->stream>>>(a);
    }
    h->launches += 1;
    return cudaGetLastError();
}

}  // namespace knnd
