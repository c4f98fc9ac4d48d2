// merge.cu -- the bounded top-K update of one round (Sec. 3.1 "Update",
// Sec. 4.2 NavigableSet insertion): the new friend list of x is the K best,
// under (key ascending, index ascending), of its old list and the candidates
// the join appended to its bucket; duplicates and x itself never enter.
//
// One warp per point x.  The list lives in registers, entry q = lane + 32*e
// (e < NE, NE = 1 for K <= 32, 2 for K <= 64); a candidate that beats the K-th
// entry is inserted by one ballot (rank), one shuffle-up (shift) and a select;
// a ballot of index equality rejects duplicates.
//
// Every bucket entry already passed the join's filter against the old K-th
// entry, and its first word orders it like its key (u: mixed form -dot,
// FP64 form the key rounded up to FP32).  The fast path therefore ranks
// candidates with integer compares only (GB300's FP64 pipe is narrow):
//  1. each lane scans its share of the bucket, drops old friends (per-warp
//     shared-memory hash) and copies of entries it holds, keeps its R smallest
//     by u, and remembers the smallest u it pushed out;
//  2. T, an upper bound of the exact K-th key of the pool: the old K-th key,
//     or (when more than 32 candidates pass) the bound of a u below which at
//     least K distinct kept candidates lie, by K rounds of warp minimum;
//  3. if some lane pushed out an entry that could still reach T, the row is
//     listed (with T) for a second kernel, which streams its bucket again 32
//     entries at a time and keys and inserts, by the batched insertion, every
//     entry whose lower bound reaches min(T, the list's current K-th key)
//     (K > 32: one at a time, on the serial path); otherwise the kept entries
//     that can reach T get their exact key (FP64 form: stored; mixed form:
//     canonical FP64 re-score) and are inserted into the old list.
// The result equals the FP64 form's bit for bit.
#include <math_constants.h>

#include <algorithm>

#include "knnd_internal.cuh"

namespace knnd {

// Exact FP64 keys as order-preserving 64-bit integers, so that the list's
// comparisons run on the integer pipe (GB300's FP64 pipe is narrow).  -0 is
// mapped to +0 so that equal keys stay equal.
__device__ __forceinline__ uint64_t dkey(double d)
{
    uint64_t b = (uint64_t)__double_as_longlong(d);
    if (b == 0x8000000000000000ull) b = 0;
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double from_dkey(uint64_t s)
{
    return __longlong_as_double((long long)((s & 0x8000000000000000ull) ? (s & 0x7fffffffffffffffull) : ~s));
}

__device__ __forceinline__ bool lex_less_u(uint64_t ka, int ia, uint64_t kb, int ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

template <int NE>
struct WarpList {
    uint64_t k[NE];  // dkey of the exact key
    int i[NE];
    int old[NE];

    __device__ __forceinline__ void kth(int K, uint64_t &kk, int &ik) const {
        const int e = (K - 1) >> 5, src = (K - 1) & 31;
        uint64_t kv = k[0];
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
    __device__ __forceinline__ void insert(int K, int lane, uint64_t ck, int ci, int cold) {
        int p = 0;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const bool less = (lane + 32 * e < K) && lex_less_u(k[e], i[e], ck, ci);
            p += __popc(__ballot_sync(0xffffffffu, less));
        }
        uint64_t uk[NE];
        int ui[NE], uo[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            uk[e] = __shfl_up_sync(0xffffffffu, k[e], 1);
            ui[e] = __shfl_up_sync(0xffffffffu, i[e], 1);
            uo[e] = __shfl_up_sync(0xffffffffu, old[e], 1);
        }
#pragma unroll
        for (int e = NE - 1; e >= 1; --e) {  // lane 0 of slot e takes lane 31 of slot e-1
            const uint64_t ck2 = __shfl_sync(0xffffffffu, k[e - 1], 31);
            const int ci2 = __shfl_sync(0xffffffffu, i[e - 1], 31);
            const int co2 = __shfl_sync(0xffffffffu, old[e - 1], 31);
            if (lane == 0) {
                uk[e] = ck2;
                ui[e] = ci2;
                uo[e] = co2;
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
    // insert (ck, ci) if it beats the K-th entry and is not listed yet
    __device__ __forceinline__ void offer(int K, int lane, uint64_t ck, int ci, uint64_t &kk, int &ik) {
        if (!lex_less_u(ck, ci, kk, ik)) return;
        if (contains(K, lane, ci)) return;
        insert(K, lane, ck, ci, 0);
        kth(K, kk, ik);
    }
};

struct MergeArgs {
    int64_t n;
    int K;
    int MP;
    int M2;  // double2 elements holding the m coordinates, (m + 1) / 2: the re-score skips the rest of the padding
    // the rows merged (read) and the rows written; in_flag marks entries already new
    // against the graph of the round's start (the second phase of a split round),
    // or NULL (every entry read is old); count: add the new entries to the update count
    const int32_t *in_idx;
    const double *in_key;
    const uint8_t *in_flag;
    int32_t *idx;
    double *key;
    uint8_t *flag;
    int count;
    const int64_t *cof_off;
    const int32_t *bcnt;
    const int2 *bent;
    const double *bkey;
    const double *X64;
    const double *L64;
    const double *negH;
    const double *Ex;
    int64_t *cnt;
    int32_t *err;
    int32_t *fb_list;   // rows left to the second kernel
    int32_t *fb_count;
    double *fb_T;       // per row: the upper bound T of its K-th key the fast path found (K <= 32)
    unsigned long long *queue;  // the work queue's counter: rows claimed so far (zeroed per launch)
    InstView iv;
};

// Several instances: a row's counts go to its instance at once.
__device__ __forceinline__ void flush_row_counts(const MergeArgs &a, int64_t x, int &newcount, long long &rescored,
                                                 long long &fallbacks)
{
    if (!a.iv.of) return;
    const int nc = __reduce_add_sync(0xffffffffu, newcount);
    long long rs = rescored, fb = fallbacks;
    for (int o = 16; o > 0; o >>= 1) {
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
        fb += __shfl_xor_sync(0xffffffffu, fb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        int64_t *c = a.iv.cnt + (int64_t)a.iv.of[x] * kCntNum;
        if (nc && a.count) atomicAdd((unsigned long long *)&c[kCntUpdates], (unsigned long long)nc);
        if (rs) atomicAdd((unsigned long long *)&c[kCntRescored], (unsigned long long)rs);
        if (fb) atomicAdd((unsigned long long *)&c[kCntFallback], (unsigned long long)fb);
    }
    newcount = 0;
    rescored = 0;
    fallbacks = 0;
}

template <int NE>
__device__ __forceinline__ void write_row(const MergeArgs &a, int64_t x, int lane, const WarpList<NE> &X,
                                          int &newcount)
{
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int q = lane + 32 * e;
        if (q < a.K) {
            a.idx[x * a.K + q] = X.i[e];
            a.key[x * a.K + q] = from_dkey(X.k[e]);
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
            X.k[e] = dkey(a.in_key[x * a.K + q]);
            X.i[e] = a.in_idx[x * a.K + q];
            X.old[e] = a.in_flag ? (a.in_flag[x * a.K + q] ? 0 : 1) : 1;
        } else {
            X.k[e] = 0;
            X.i[e] = -1;
            X.old[e] = 1;
        }
    }
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

__device__ __forceinline__ void flush_counts(const MergeArgs &a, int newcount, long long rescored,
                                             long long fallbacks, long long survivors = 0)
{
    if ((threadIdx.x & 31) == 0 && survivors)
        atomicAdd((unsigned long long *)&a.cnt[kCntSurvivors], (unsigned long long)survivors);
    newcount = __reduce_add_sync(0xffffffffu, newcount);
    for (int o = 16; o > 0; o >>= 1) {
        rescored += __shfl_xor_sync(0xffffffffu, rescored, o);
        fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (newcount && a.count) atomicAdd((unsigned long long *)&a.cnt[kCntUpdates], (unsigned long long)newcount);
        if (rescored) atomicAdd((unsigned long long *)&a.cnt[kCntRescored], (unsigned long long)rescored);
        if (fallbacks) atomicAdd((unsigned long long *)&a.cnt[kCntFallback], (unsigned long long)fallbacks);
    }
}

// Canonical FP64 key of (x, y): the same fma chain as the join and the
// initial graph.  TRIM (the one-entry-per-lane lists, K <= 32): the chain
// stops at the first even count >= m, since the padding terms past m are exact
// no-ops (0 * 0 added) and FP64 issue is scarce on this GPU; otherwise it runs
// over the padded width, eight coordinates per step (fewer registers).
template <bool TRIM>
__device__ __forceinline__ double rescore(const MergeArgs &a, int64_t x, int y, double nh)
{
    const double2 *xr = reinterpret_cast<const double2 *>(a.X64 + x * a.MP);
    const double2 *lr = reinterpret_cast<const double2 *>(a.L64 + (int64_t)y * a.MP);
    double acc = 0.0;
    if (TRIM) {
#pragma unroll 4
        for (int i2 = 0; i2 < a.M2; ++i2) {
            const double2 p = __ldg(xr + i2), q = __ldg(lr + i2);
            acc = __fma_rn(p.x, q.x, acc);
            acc = __fma_rn(p.y, q.y, acc);
        }
    } else {
        for (int i8 = 0; i8 < a.MP / 8; ++i8) {
            double2 p[4], q[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                p[t] = __ldg(xr + 4 * i8 + t);
                q[t] = __ldg(lr + 4 * i8 + t);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                acc = __fma_rn(p[t].x, q[t].x, acc);
                acc = __fma_rn(p[t].y, q[t].y, acc);
            }
        }
    }
    return nh - acc;
}

// key(x, y) under the comparator CMP: KL negH(x) - <x, log y>; reverse KL the
// same chain with the roles swapped; squared Euclidean (|x|^2 - 2 <x, y>) + |y|^2
// (the tables then hold the coordinates and the squared norms).  nh: negH(x).
template <int CMP, bool TRIM>
__device__ __forceinline__ double rescore_dir(const MergeArgs &a, int64_t x, int y, double nh)
{
    if (CMP == KNND_CMP_KL_REVERSE) return rescore<TRIM>(a, (int64_t)y, (int)x, a.negH[y]);
    if (CMP == KNND_CMP_SQEUCLIDEAN) return (a.negH[x] + 2.0 * rescore<TRIM>(a, x, y, 0.0)) + a.negH[y];
    return rescore<TRIM>(a, x, y, nh);
}

// ------------------------------------------------------------------ old-list set
// Per-warp open-addressing set of the row's old friend indices in shared
// memory (kHashSlots >= 2 K): about one probe per lookup.
constexpr int kHashSlots = 128;

__device__ __forceinline__ unsigned hash_slot(int y) { return ((unsigned)y * 0x9E3779B1u) >> 25; }

template <int NE>
__device__ __forceinline__ void hash_fill(int *tab, int lane, int K, const WarpList<NE> &X)
{
    for (int s = lane; s < kHashSlots; s += 32) tab[s] = -1;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int y = X.i[e];
        if (lane + 32 * e < K && y >= 0) {
            unsigned sl = hash_slot(y);
            for (int t = 0; t < kHashSlots; ++t) {
                const int prev = atomicCAS(&tab[sl], -1, y);
                if (prev == -1 || prev == y) break;
                sl = (sl + 1) & (kHashSlots - 1);
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ bool hash_has(const int *tab, int y)
{
    unsigned sl = hash_slot(y);
    for (int t = 0; t < kHashSlots; ++t) {
        const int v = tab[sl];
        if (v == y) return true;
        if (v == -1) return false;
        sl = (sl + 1) & (kHashSlots - 1);
    }
    return false;
}

// ------------------------------------------------------------------ key bounds
// Bounds of the exact key of an entry from its u, and the u-threshold of
// "lower bound <= T".
template <bool MIXED>
struct Bounds {
    double nh, E;
    __device__ __forceinline__ double upper(float u) const { return MIXED ? (nh + (double)u) + E : (double)u; }
    // every entry whose lower bound is <= T has u <= u_reach(T)
    __device__ __forceinline__ float u_reach(double T) const {
        return MIXED ? __double2float_ru((T - nh) + E) : __double2float_ru(T);
    }
};

// ------------------------------------------------------------------ serial path
// Candidates are inserted one at a time.  Used for rows the fast path cannot
// settle.  Mixed form: pass A keeps the K best upper bounds (threshold T),
// pass B re-scores every candidate whose lower bound reaches T.
template <int NE, bool MIXED, int CMP>
__device__ void serial_row(const MergeArgs &a, int64_t x, int lane, WarpList<NE> &X, const int *tab, int64_t base,
                           int cnt, const Bounds<MIXED> &B, long long &rescored)
{
    const int K = a.K;
    double T = CUDART_INF;
    if (MIXED) {
        WarpList<NE> A = X;
        uint64_t tk;
        int ti;
        A.kth(K, tk, ti);
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const bool has = c0 + lane < cnt;
            uint64_t ub = ~0ull;
            int ci = -1;
            if (has) {
                const int2 en = a.bent[base + c0 + lane];
                ub = dkey(B.upper(from_sortable_bits((uint32_t)en.x)));
                ci = en.y;
            }
            const bool take = has && ci >= 0 && ci < a.n && !hash_has(tab, ci);
            unsigned mask = __ballot_sync(0xffffffffu, take && lex_less_u(ub, ci, tk, ti));
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                A.offer(K, lane, __shfl_sync(0xffffffffu, ub, src), __shfl_sync(0xffffffffu, ci, src), tk, ti);
            }
        }
        T = from_dkey(tk);
    }
    uint64_t xk;
    int xi;
    X.kth(K, xk, xi);
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const bool has = c0 + lane < cnt;
        int ci = -1;
        float u = 0.f;
        if (has) {
            const int2 en = a.bent[base + c0 + lane];
            u = from_sortable_bits((uint32_t)en.x);
            ci = en.y;
        }
        bool want = has && ci >= 0 && ci < a.n && !hash_has(tab, ci);
        if (MIXED) want = want && u <= B.u_reach(fmin(T, from_dkey(xk)));
        uint64_t k = 0;
        if (want) {
            if (MIXED) {
                k = dkey(rescore_dir<CMP, NE == 1>(a, x, ci, B.nh));
                rescored += 1;
            } else {
                k = dkey(a.bkey[base + c0 + lane]);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, want);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            X.offer(K, lane, __shfl_sync(0xffffffffu, k, src), __shfl_sync(0xffffffffu, ci, src), xk, xi);
        }
    }
}

// ------------------------------------------------------------------ fast path
// A lane's R smallest candidates by u (ties in arrival order), held in
// registers as 32-bit fields: the threshold extraction reads u alone, so the
// list needs no 64-bit (u, index) keys.
template <int R>
struct LaneTop {
    uint32_t u[R];  // sortable u, ascending; ~0 = empty
    int y[R];       // candidate index, -1 = empty
    int pos[R];     // bucket slot of the entry
    uint32_t drop;  // smallest sortable u pushed out (~0 = none)

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            u[r] = 0xffffffffu;
            y[r] = -1;
            pos[r] = 0;
        }
        drop = 0xffffffffu;
    }
    __device__ __forceinline__ void push(uint32_t pu, int py, int ps) {
        if (pu >= u[R - 1]) {
            drop = min(drop, pu);
            return;
        }
        // a copy of an entry this lane already holds (same u, same index) adds
        // nothing; the last entry's u is above pu, so no copy sits there
        bool dup = false;
#pragma unroll
        for (int r = 0; r < R - 1; ++r) dup |= (u[r] == pu) & (y[r] == py);
        if (dup) return;
        drop = min(drop, u[R - 1]);  // the last entry leaves (~0 when the list was not full)
        // entry r of the new list: the old entry r - 1 when pu goes before it,
        // else pu when it goes before the old entry r, else the old entry r
        bool c[R];
#pragma unroll
        for (int r = 0; r < R; ++r) c[r] = pu < u[r];
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            const int rm = r > 0 ? r - 1 : 0;
            const bool before = r > 0 && c[rm];
            u[r] = before ? u[rm] : (c[r] ? pu : u[r]);
            y[r] = before ? y[rm] : (c[r] ? py : y[r]);
            pos[r] = before ? pos[rm] : (c[r] ? ps : pos[r]);
        }
    }
};

// Per-warp scratch of the batched insertion (K <= 32).
struct BatchScratch {
    uint64_t xk[32], ck[32], mk[32];
    int xi[32], ci[32], mi[32], mo[32];
};

// Inserts up to 32 candidates at once (one per lane: key k, index ci, when
// `has`) into the sorted list X of K <= 32 entries: candidates that cannot
// beat the K-th entry are dropped; the rest are sorted by (key, index) with a
// warp bitonic network, copies of one candidate and copies of listed entries
// are dropped, and each entry's place in the merged list is its own index
// plus its rank in the other list (binary search in shared memory).  Same
// result as offering the candidates one by one.
__device__ __forceinline__ void insert_batch(WarpList<1> &X, int K, int lane, uint64_t k, int ci, bool has,
                                             uint64_t &xk, int &xi, BatchScratch &sb)
{
    const unsigned FULL = 0xffffffffu;
    bool v = has && lex_less_u(k, ci, xk, xi);
    const unsigned vm0 = __ballot_sync(FULL, v);
    if (!vm0) return;
    // lanes above the highest candidate hold +inf, so the stages that sort blocks of up
    // to the first power of two above it sort every candidate (in the lowest block)
    const int top = 31 - __clz(vm0);
    uint64_t ck = v ? k : ~0ull;
    int cj = v ? ci : 0x7fffffff;
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
        if ((kk >> 1) > top) break;
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const uint64_t ok = __shfl_xor_sync(FULL, ck, j);
            const int oj = __shfl_xor_sync(FULL, cj, j);
            const bool keep_min = ((lane & kk) == 0) == ((lane & j) == 0);
            const bool take = keep_min ? lex_less_u(ok, oj, ck, cj) : lex_less_u(ck, cj, ok, oj);
            if (take) {
                ck = ok;
                cj = oj;
            }
        }
    }
    const int pj = __shfl_up_sync(FULL, cj, 1);
    v = ck != ~0ull && !(lane > 0 && pj == cj);  // one index, one key: copies are adjacent
    if (lane < K) {
        sb.xk[lane] = X.k[0];
        sb.xi[lane] = X.i[0];
    }
    __syncwarp();
    int rc = 0;  // listed entries before the candidate
    if (v) {
        int lo = 0, hi = K;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lex_less_u(sb.xk[mid], sb.xi[mid], ck, cj)) lo = mid + 1;
            else hi = mid;
        }
        rc = lo;
        if (lo < K && sb.xi[lo] == cj) v = false;  // already listed
    }
    const unsigned vm = __ballot_sync(FULL, v);
    const int L = __popc(vm), cpos = __popc(vm & lanemask_lt());
    if (v) {
        sb.ck[cpos] = ck;
        sb.ci[cpos] = cj;
    }
    __syncwarp();
    if (lane < K) {  // listed entry: its index plus the candidates before it
        int lo = 0, hi = L;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (lex_less_u(sb.ck[mid], sb.ci[mid], X.k[0], X.i[0])) lo = mid + 1;
            else hi = mid;
        }
        const int pos = lane + lo;
        if (pos < K) {
            sb.mk[pos] = X.k[0];
            sb.mi[pos] = X.i[0];
            sb.mo[pos] = X.old[0];
        }
    }
    if (v && cpos + rc < K) {
        sb.mk[cpos + rc] = ck;
        sb.mi[cpos + rc] = cj;
        sb.mo[cpos + rc] = 0;
    }
    __syncwarp();
    if (lane < K) {
        X.k[0] = sb.mk[lane];
        X.i[0] = sb.mi[lane];
        X.old[0] = sb.mo[lane];
    }
    __syncwarp();
    X.kth(K, xk, xi);
}

// Rows of K <= 32 whose kept entries do not cover every entry that can reach
// T.  The bucket is scanned 32 entries at a time; the entries whose lower
// bound reaches min(T, the list's K-th key) are compacted into `pend` (kPend
// per warp, by ballot), and each time it holds at least 32 (and at the end)
// they are keyed and inserted 32 at a time by the batched insertion, skipping
// those that the list has left behind meanwhile.  (The pending list is drained
// whenever the next 32 entries might not fit, and at the end.)
constexpr int kPend = 256;

template <bool MIXED, int CMP>
__device__ __forceinline__ void stream_row(const MergeArgs &a, int64_t x, int lane, WarpList<1> &X, const int *tab,
                                        int64_t base, int cnt, const Bounds<MIXED> &B, double T, long long &rescored,
                                        BatchScratch &sb, int2 *pend)
{
    const int K = a.K;
    const unsigned lt = lanemask_lt();
    uint64_t xk;
    int xi;
    X.kth(K, xk, xi);
    int np = 0;  // entries pending in pend: (index, bucket slot)
    auto drain = [&]() {
        for (int c0 = 0; c0 < np; c0 += 32) {
            const bool has = c0 + lane < np;
            int ci = -1;
            uint64_t k = ~0ull;
            bool want = false;
            if (has) {
                const int2 e = pend[c0 + lane];
                ci = e.x;
                const uint32_t u = (uint32_t)a.bent[base + e.y].x;
                want = u <= sortable_bits(B.u_reach(fmin(T, from_dkey(xk))));
                if (want) {
                    if (MIXED) {
                        k = dkey(rescore_dir<CMP, true>(a, x, ci, B.nh));
                        rescored += 1;
                    } else {
                        k = dkey(a.bkey[base + e.y]);
                    }
                }
            }
            insert_batch(X, K, lane, k, ci, want, xk, xi, sb);
        }
        np = 0;
        __syncwarp();
    };
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const bool has = c0 + lane < cnt;
        const int2 en = has ? a.bent[base + c0 + lane] : make_int2(0, -1);
        const int ci = en.y;
        const uint32_t lim = sortable_bits(B.u_reach(fmin(T, from_dkey(xk))));
        const bool want = has && ci >= 0 && ci < a.n && (uint32_t)en.x <= lim && !hash_has(tab, ci);
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (np + __popc(m) > kPend) drain();
        if (want) pend[np + __popc(m & lt)] = make_int2(ci, c0 + lane);
        np += __popc(m);
        __syncwarp();
    }
    drain();
}

template <int NE, int R, bool MIXED, int CMP>
__device__ bool fast_row(const MergeArgs &a, int64_t x, int lane, WarpList<NE> &X, const int *tab, int2 *live_list,
                         int64_t base, int cnt, const Bounds<MIXED> &B, long long &rescored, BatchScratch &sb)
{
    const int K = a.K;
    LaneTop<R> L;
    L.init();
    int passing = 0;
    for (int c0 = lane; c0 < cnt; c0 += 4 * 32) {
        int2 en[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)  // four independent loads in flight per lane
            en[t] = (c0 + 32 * t < cnt) ? a.bent[base + c0 + 32 * t] : make_int2(0, -1);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if ((uint32_t)en[t].y >= (uint32_t)a.n || hash_has(tab, en[t].y)) continue;  // also y < 0
            passing += 1;
            L.push((uint32_t)en[t].x, en[t].y, c0 + 32 * t);
        }
    }
    const int P = __reduce_add_sync(0xffffffffu, passing);
    if (P == 0) return true;
    uint64_t T0;
    int Ti;
    X.kth(K, T0, Ti);
    double T = from_dkey(T0);
    if (P > 32) {
        // the K-th smallest u among the lanes' lists, one u value per step: the warp
        // minimum of the heads' u (one single-instruction warp reduction), and every
        // lane whose head has that u pops it.  The steps spent at one value w number
        // the most entries of u = w that one lane holds, never more than the distinct
        // candidates of u = w (a lane holds no candidate twice), so after K steps at
        // least K distinct candidates have u <= mu: T bounds the K-th key from above
        int popped = 0, count = 0;
        uint32_t mu = 0xffffffffu;
        while (count < K) {
            uint32_t hu = 0xffffffffu;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r == popped) hu = L.u[r];
            mu = __reduce_min_sync(0xffffffffu, hu);
            if (mu == 0xffffffffu) break;  // every list exhausted
            popped += (hu == mu) ? 1 : 0;
            count += 1;
        }
        if (count == K) T = fmin(T, B.upper(from_sortable_bits(mu)));
    }
    const uint32_t reach = sortable_bits(B.u_reach(T));
    if (__any_sync(0xffffffffu, L.drop <= reach)) {
        if (lane == 0) a.fb_T[x] = T;  // the second kernel streams the bucket against it
        return false;
    }
    // compact the entries that can reach T, then key them 32 at a time
    const unsigned lt = lanemask_lt();
    int nlive = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool live = L.y[r] >= 0 && L.u[r] <= reach;
        const unsigned mask = __ballot_sync(0xffffffffu, live);
        if (live) live_list[nlive + __popc(mask & lt)] = make_int2(L.y[r], L.pos[r]);
        nlive += __popc(mask);
    }
    __syncwarp();
    uint64_t xk;
    int xi;
    X.kth(K, xk, xi);
    for (int c0 = 0; c0 < nlive; c0 += 32) {
        const bool has = c0 + lane < nlive;
        int ci = -1;
        uint64_t k = ~0ull;
        if (has) {
            const int2 e = live_list[c0 + lane];
            ci = e.x;
            if (MIXED) {
                k = dkey(rescore_dir<CMP, NE == 1>(a, x, ci, B.nh));
                rescored += 1;
            } else {
                k = dkey(a.bkey[base + e.y]);
            }
        }
        if constexpr (NE == 1) {
            insert_batch(X, K, lane, k, ci, has, xk, xi, sb);
        } else {
            unsigned mask = __ballot_sync(0xffffffffu, has);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                X.offer(K, lane, __shfl_sync(0xffffffffu, k, src), __shfl_sync(0xffffffffu, ci, src), xk, xi);
            }
        }
    }
    __syncwarp();
    return true;
}

// CMP: the comparator (KNND_CMP_*) the mixed forms re-score with; the entries'
// u orders candidates like key - ro(x), ro = negH(x) for KL, |x|^2 for squared
// Euclidean, 0 for reverse KL.
// Rows per claim of the work queue: 4 measured 5 % faster than 16 at n = 4e5,
// d = 20, K = 20 (the last claims finish closer together); 32 was slower.
constexpr int kRowChunk = 4;

template <int NE, int R, bool MIXED, int CMP>
__global__ void __launch_bounds__(256) merge_kernel(MergeArgs a)
{
    __shared__ int s_hash[8][kHashSlots];
    __shared__ int2 s_live[8][32 * R];
    __shared__ BatchScratch s_batch[NE == 1 ? 8 : 1];
    const int lane = threadIdx.x & 31;
    const int K = a.K;
    int *tab = s_hash[threadIdx.x >> 5];
    int2 *live_list = s_live[threadIdx.x >> 5];
    int newcount = 0;
    long long rescored = 0, fallbacks = 0, survivors = 0;
    // rows from the work queue: chunks of kRowChunk consecutive rows, each claimed
    // by one atomicAdd as the warp reaches it (rows differ widely in cost)
    int64_t x = 0, xend = 0;
    auto claim = [&]() {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.queue, (unsigned long long)kRowChunk);
        t = __shfl_sync(0xffffffffu, t, 0);
        x = (int64_t)t;
        xend = min(x + kRowChunk, a.n);
    };
    claim();
    for (; x < a.n; ++x) {
        if (x >= xend) {
            claim();
            if (x >= a.n) break;
        }
        if (!a.iv.live(x)) continue;  // row of a stopped instance (batched form)
        WarpList<NE> X;
        load_row(a, x, lane, X);
        const int64_t base = (int64_t)K * K * x + (int64_t)(K + 1) * a.cof_off[x];
        const int cnt = bucket_count(a, x);
        survivors += cnt;
        if (cnt > 0) {
            Bounds<MIXED> B;
            B.nh = (MIXED && CMP != KNND_CMP_KL_REVERSE) ? a.negH[x] : 0.0;
            B.E = MIXED ? a.Ex[x] : 0.0;
            hash_fill(tab, lane, K, X);
            if (!fast_row<NE, R, MIXED, CMP>(a, x, lane, X, tab, live_list, base, cnt, B, rescored,
                                        s_batch[NE == 1 ? (threadIdx.x >> 5) : 0])) {
                // the row stays as it is here; merge_fallback_kernel finishes it
                if (lane == 0) {
                    a.fb_list[atomicAdd(a.fb_count, 1)] = (int32_t)x;
                    fallbacks += 1;  // once per row (the counts are summed over the lanes)
                }
                flush_row_counts(a, x, newcount, rescored, fallbacks);
                continue;
            }
        }
        write_row(a, x, lane, X, newcount);
        flush_row_counts(a, x, newcount, rescored, fallbacks);
    }
    flush_counts(a, newcount, rescored, fallbacks, survivors);
}

// Rows the fast path could not settle, one warp each, on the serial path.
template <int NE, bool MIXED, int CMP>
__global__ void __launch_bounds__(256, 2) merge_fallback_kernel(MergeArgs a)
{
    __shared__ int s_hash[8][kHashSlots];
    __shared__ BatchScratch s_batch[NE == 1 ? 8 : 1];
    __shared__ int2 s_pend[NE == 1 ? 8 : 1][NE == 1 ? kPend : 1];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int K = a.K;
    int *tab = s_hash[threadIdx.x >> 5];
    int newcount = 0;
    long long rescored = 0;
    const int nfb = *a.fb_count;
    for (int f = blockIdx.x * wpb + (threadIdx.x >> 5); f < nfb; f += gridDim.x * wpb) {
        const int64_t x = a.fb_list[f];
        WarpList<NE> X;
        load_row(a, x, lane, X);
        const int64_t base = (int64_t)K * K * x + (int64_t)(K + 1) * a.cof_off[x];
        const int cnt = bucket_count(a, x);
        Bounds<MIXED> B;
        B.nh = (MIXED && CMP != KNND_CMP_KL_REVERSE) ? a.negH[x] : 0.0;
        B.E = MIXED ? a.Ex[x] : 0.0;
        hash_fill(tab, lane, K, X);
        if constexpr (NE == 1)  // the threshold T the fast path found for the row
            stream_row<MIXED, CMP>(a, x, lane, X, tab, base, cnt, B, a.fb_T[x], rescored, s_batch[threadIdx.x >> 5],
                                   s_pend[threadIdx.x >> 5]);
        else
            serial_row<NE, MIXED, CMP>(a, x, lane, X, tab, base, cnt, B, rescored);
        write_row(a, x, lane, X, newcount);
        long long nofb = 0;
        flush_row_counts(a, x, newcount, rescored, nofb);
    }
    flush_counts(a, newcount, rescored, 0);
}

template <int NE, int R, bool MIXED, int CMP>
static void launch_merge_pair(knnd_handle *h, const MergeArgs &a, int64_t grid, unsigned fgrid, int threads)
{
    merge_kernel<NE, R, MIXED, CMP><<<(unsigned)grid, threads, 0, h->stream>>>(a);
    merge_fallback_kernel<NE, MIXED, CMP><<<fgrid, threads, 0, h->stream>>>(a);
}

cudaError_t launch_merge(knnd_handle *h, int32_t *idx, double *key, uint8_t *newflag)
{
    return launch_merge_from(h, idx, key, nullptr, idx, key, newflag, true);
}

cudaError_t launch_merge_from(knnd_handle *h, const int32_t *in_idx, const double *in_key, const uint8_t *in_flag,
                              int32_t *idx, double *key, uint8_t *newflag, bool count)
{
    MergeArgs a;
    a.n = h->n;
    a.K = h->K;
    a.MP = h->MP;
    a.M2 = (h->m + 1) / 2;
    a.in_idx = in_idx;
    a.in_key = in_key;
    a.in_flag = in_flag;
    a.idx = idx;
    a.key = key;
    a.flag = newflag;
    a.count = count ? 1 : 0;
    a.cof_off = h->cof_off;
    a.bcnt = h->bcnt;
    a.bent = h->bent;
    a.bkey = h->bkey;
    a.X64 = h->X64;
    a.L64 = h->L64;
    a.negH = h->negH;
    a.Ex = h->Ex;
    a.cnt = h->cnt;
    a.err = h->err;
    const int threads = 256;
    const int64_t need = (h->n + threads / 32 - 1) / (threads / 32);
    const int64_t grid = std::min<int64_t>(need, (int64_t)h->num_sms * 8);
    a.fb_list = h->fb_list;
    a.fb_count = h->fb_count;
    a.fb_T = h->fb_T;
    a.queue = h->join_queue + 1;
    cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), h->stream);
    a.iv = h->iv;
    cudaMemsetAsync(h->fb_count, 0, sizeof(int32_t), h->stream);
    const bool fp64 = h->prec == KNND_PREC_FP64;
    // the inner product re-scores with the KL chain (negH = 0, L = coordinates)
    const bool kl_form = h->prm.comparator == KNND_CMP_KL || h->prm.comparator == KNND_CMP_INNER;
    const unsigned fgrid = (unsigned)h->num_sms * 2;
    // the FP64 form's keys come from the join (no re-score): one instance serves every comparator
    if (h->K <= 32 && h->merge_keep == 8) {  // more candidates kept per lane: fewer rows need the second kernel
        if (fp64) launch_merge_pair<1, 8, false, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (kl_form) launch_merge_pair<1, 8, true, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (h->prm.comparator == KNND_CMP_KL_REVERSE)
            launch_merge_pair<1, 8, true, KNND_CMP_KL_REVERSE>(h, a, grid, fgrid, threads);
        else launch_merge_pair<1, 8, true, KNND_CMP_SQEUCLIDEAN>(h, a, grid, fgrid, threads);
    } else if (h->K <= 32) {
        if (fp64) launch_merge_pair<1, 4, false, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (kl_form) launch_merge_pair<1, 4, true, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (h->prm.comparator == KNND_CMP_KL_REVERSE)
            launch_merge_pair<1, 4, true, KNND_CMP_KL_REVERSE>(h, a, grid, fgrid, threads);
        else launch_merge_pair<1, 4, true, KNND_CMP_SQEUCLIDEAN>(h, a, grid, fgrid, threads);
    } else {
        if (fp64) launch_merge_pair<2, 8, false, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (kl_form) launch_merge_pair<2, 8, true, KNND_CMP_KL>(h, a, grid, fgrid, threads);
        else if (h->prm.comparator == KNND_CMP_KL_REVERSE)
            launch_merge_pair<2, 8, true, KNND_CMP_KL_REVERSE>(h, a, grid, fgrid, threads);
        else launch_merge_pair<2, 8, true, KNND_CMP_SQEUCLIDEAN>(h, a, grid, fgrid, threads);
    }
    h->launches += 2;
    return cudaGetLastError();
}

}  // namespace knnd
