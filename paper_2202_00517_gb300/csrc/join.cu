// join.cu -- the local join of one round (Sec. 3.1 "Meet", Sec. 4.2
// proposeNewFriendSet), organised around hubs.
//
// Every pair the pool of Sec. 3.1 contains is met at exactly one hub role:
//   x in coF(v), y in F(v)   <=>  y is a friend of a friend of x
//   x in F(v),   y in F(v)   <=>  y is a friend of a co-friend of x
//   x in F(v),   y = v       <=>  y is a co-friend of x
// so hub v's tile is rows R_v = F(v) + coF(v) against columns F(v), plus the
// column v for the rows of F(v).  The tile is a small dense contraction of the
// rows' coordinates with the columns' log table: key(x, y) = negH(x) - <x, L(y)>.
//
// One warp per hub (for the inner product, hubs with very many rows go to a
// second pass that splits their rows over several warps).  Columns' log rows
// sit in registers (FP64 form: lane j holds column j; mixed form: a lane holds
// a column pair of one row group); the rows are staged 32 at a time in shared
// memory.  A pair that can still beat row x's current K-th entry is appended to
// x's bucket (capacity K*K + (K+1)*indeg(x), so it cannot overflow): one
// atomicAdd per (hub, row) reserves the row's slots, then the warp writes the
// survivors consecutively.
//
// FP64 form: key in FP64, exact filter (key, y) < (tau_x, idxK_x); the entry
// stores the key (bkey) and its FP32 round-up.
// Mixed form: FP32 dot with FP32 accumulation; the pair is rejected only when
// dot + E_x < negH_x - tau_x, i.e. when it provably cannot beat the K-th
// entry (phi_x = that threshold, rounded down); the entry stores -dot and the
// merge re-scores in FP64.  Either way the entry's first word orders the
// candidates like their keys (sortable float bits).
#include <algorithm>

#include "knnd_internal.cuh"

namespace knnd {

struct JoinArgs {
    int64_t n;
    int64_t h_lo, h_hi;  // the hubs this launch takes: [h_lo, h_hi), those of phase `phase` (in_phase)
    int phase, split_den;
    // heavy hubs (more than kHeavyRows rows): the main pass skips them and a second
    // pass spreads their rows over the grid as items (hub, group of kItemRows rows)
    const int2 *items;        // NULL: no heavy pass
    const int32_t *nitems;
    int heavy_pass;           // 1: this launch runs the items
    int K;
    const int32_t *idx;
    const int64_t *cof_off;
    const int32_t *cof;
    const float *X32;
    const float *L32;
    const double *X64;
    const double *L64;
    const double *negH;
    const double *tau;
    const int32_t *idxK;
    const RowMeta *meta;
    int32_t *bcnt;
    int2 *bent;
    double *bkey;
    int32_t *err;
    int debug;
    InstView iv;
    // incremental proposals: flags of G_{r-1} (n x K) and of the coF entries,
    // or NULL (every pair proposed).  A pair met only through arcs whose flag
    // is 0 was in the previous round's pool and is not proposed again.
    const uint8_t *flag;
    const uint8_t *cof_new;
    // comparator (KNND_CMP_*).  Reverse KL (key(x, y) = negH(y) - <y, log x>): the
    // launch swaps the coordinate and log tables, so rows read log x and columns
    // read y, and the offset belongs to the column.  Squared Euclidean
    // ((|x|^2 - 2 <x, y>) + |y|^2, negH holding the squared norms): both offsets,
    // dot scale 2.  col_scale: 1 or 2; col_inv: its inverse (exact).
    int cmp;
    float col_scale;
    double col_inv;
};

// New-flag of the arc that makes row r (of hub v) a row of the tile: v -> x
// for the first K rows (x in F(v)), x -> v for the co-friend rows.
__device__ __forceinline__ int row_new(const JoinArgs &a, int64_t v, int K, int64_t c0, int64_t r)
{
    if (!a.flag) return 1;
    return r < K ? a.flag[v * K + r] : a.cof_new[c0 + (r - K)];
}

__device__ __forceinline__ bool valid_id(int64_t v, int64_t n) { return v >= 0 && v < n; }

// Comparators whose key has a per-column offset co(y) (reverse KL, squared
// Euclidean); KL and inner product have none (key = ro(x) - <R(x), C(y)>).
__host__ __device__ __forceinline__ bool has_col_offset(int cmp)
{
    return cmp == KNND_CMP_KL_REVERSE || cmp == KNND_CMP_SQEUCLIDEAN;
}

// ------------------------------------------------------------------ heavy hubs
// A hub's rows are F(v) and coF(v): K + indeg(v).  Skewed graphs (the inner
// product's, whose best matches are the few points of largest norm) give some
// hubs tens of thousands of rows, which one warp would take alone.
constexpr int kHeavyRows = 1024;
constexpr int kItemRows = 256;

// Items of the heavy pass, one thread per hub of the launch's range.
__global__ void heavy_items_kernel(JoinArgs a, int2 *items, int32_t *nitems)
{
    const int64_t v = a.h_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.h_hi || !a.iv.live(v) || !in_phase(a.iv, a.phase, a.split_den, a.n, v)) return;
    const int64_t nrows = (int64_t)a.K + (a.cof_off[v + 1] - a.cof_off[v]);
    if (nrows <= kHeavyRows) return;
    const int cnt = (int)((nrows + kItemRows - 1) / kItemRows);
    const int b = atomicAdd(nitems, cnt);
    for (int k = 0; k < cnt; ++k) items[b + k] = make_int2((int)v, k);
}

// ------------------------------------------------------------------ mixed
// Lane (g, p): column pair p (columns 2p, 2p+1; their FP32 log rows live in
// registers) of row group g; a pass scores two rows per group, 2 x G rows in
// all (G = 32 / ceil(K/2) groups; K = 20: 30 lanes busy, six rows a pass).
// Each lane reuses every coordinate it reads from shared memory for two
// columns.  The dots go to shared memory; then lane t owns row t of the chunk:
// it applies the filter, scores the co-friend pair (rows of F(v)), reserves the
// row's slots with one atomicAdd and writes its survivors.
template <int MP>
struct MixedSmem {
    static constexpr int RS = MP + 4;       // row stride of the staged coordinates (floats)
    static constexpr int X_FLOATS = 33 * RS; // 32 rows + the hub's own log row
    // dots of one row: stride K or K+1, whichever is odd (conflict-free row reads)
    static __host__ __device__ int d_stride(int K) { return (K & 1) ? K : K + 1; }
    // per warp: coordinates | dots | column ids (64) | survivor columns (32 x K bytes)
    //           | survivor prefix (32 ints) | row bases (32 int64)
    static __host__ __device__ int off_cid(int K) { return 4 * (X_FLOATS + 32 * d_stride(K)); }
    static __host__ __device__ int off_j(int K) { return off_cid(K) + 4 * 64; }
    static __host__ __device__ int off_inc(int K) { return off_j(K) + ((32 * K + 15) & ~15); }
    static __host__ __device__ int off_rb(int K) { return off_inc(K) + 4 * 32; }
    static __host__ __device__ int off_cnew(int K) { return off_rb(K) + 8 * 32; }
    static __host__ __device__ int off_hcol(int K) { return off_cnew(K) + 64; }
    static __host__ __device__ int warp_bytes(int K) { return off_hcol(K) + 4 * 64; }
};

// Resident blocks of 128 threads per SM the kernel is compiled for: the
// register budget grows with the two MP-wide column registers of each lane
// (spill-free at every MP; measured best at n = 4e5..1e6: 20 warps per SM for
// MP <= 16, 16 for MP 24..32, 8 for MP 48..96; MP = 128 scores in 32-wide
// coordinate chunks and fits 12).
__host__ __device__ constexpr int mixed_min_blocks(int MP) {
    return MP <= 16 ? 5 : (MP <= 32 ? 4 : (MP <= 96 ? 2 : 3));
}

// INC: incremental proposals (a.flag non-NULL); compiled apart so that the
// default form carries none of its state.
// COL: the comparator has a column offset (reverse KL, squared Euclidean): the
// filter threshold and the entry take RD(co(y)/s) of each column.
// PASS: 0 every hub of the launch; 1 the same, the heavy hubs left to pass 2;
// 2 the heavy pass (items instead of hubs; see heavy_items_kernel).
template <int MP, bool INC, bool COL, int PASS>
__global__ void __launch_bounds__(128, mixed_min_blocks(MP)) join_mixed_kernel(JoinArgs a)
{
    using S = MixedSmem<MP>;
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int K = a.K;
    const int DS = S::d_stride(K);
    unsigned char *wbase = reinterpret_cast<unsigned char *>(smem4) + (size_t)warp * S::warp_bytes(K);
    float *sX = reinterpret_cast<float *>(wbase);
    float *sD = sX + S::X_FLOATS;
    int *sCid = reinterpret_cast<int *>(wbase + S::off_cid(K));
    unsigned char *sJ = wbase + S::off_j(K);
    int *sInc = reinterpret_cast<int *>(wbase + S::off_inc(K));
    int64_t *sRB = reinterpret_cast<int64_t *>(wbase + S::off_rb(K));
    unsigned char *sCnew = wbase + S::off_cnew(K);  // new-flags of the columns
    float *sH = reinterpret_cast<float *>(wbase + S::off_hcol(K));  // COL: RD(co(y) / s) of the columns
    const int64_t n = a.n;
    const int npairs = (K + 1) >> 1;
    const int G = 32 / npairs;                 // row groups
    const int g = lane / npairs, pr = lane - g * npairs;
    const bool active = g < G;
    const int cA = 2 * pr, cB = 2 * pr + 1;     // this lane's columns

    // Short rows and K <= 32: the hub's ids come in one step (the columns F(v) are
    // also its first K rows), then its column log rows and its first chunk of
    // rows in a second, all in flight together; the columns are staged in the dot
    // buffer (stride CS) until each lane has read its two.  cof_off is read one
    // hub ahead.
    // The heavy pass takes items (hub, row group) instead of hubs, one per warp,
    // and runs the general path.
    constexpr bool heavy = PASS == 2;
    const bool fast = MP <= 32 && K <= 32 && !heavy;
    const int CS = (K * (MP + 4) <= 32 * DS) ? MP + 4 : MP;
    // t: the hub (passes 0, 1) or the item (pass 2); cof_off is read one ahead
    const int64_t tstep = (int64_t)gridDim.x * wpb;
    const int64_t tend = heavy ? (int64_t)*a.nitems : a.h_hi;
    int64_t t = (heavy ? 0 : a.h_lo) + (int64_t)blockIdx.x * wpb + warp;
    int64_t vn = 0;  // pass 2: the next item's hub
    int64_t nc0 = 0, nc1 = 0;
    if (t < tend) {
        if (heavy) vn = a.items[t].x;
        nc0 = a.cof_off[heavy ? vn : t];
        nc1 = a.cof_off[(heavy ? vn : t) + 1];
    }
    for (; t < tend; t += tstep) {
        const int64_t v = heavy ? vn : t;
        const int64_t c0 = nc0, c1 = nc1;
        const int grp = heavy ? a.items[t].y : 0;
        if (t + tstep < tend) {
            if (heavy) vn = a.items[t + tstep].x;
            nc0 = a.cof_off[heavy ? vn : t + tstep];
            nc1 = a.cof_off[(heavy ? vn : t + tstep) + 1];
        }
        if (!heavy) {
            if (!a.iv.live(v)) continue;  // hub of a stopped instance (batched form)
            if (!in_phase(a.iv, a.phase, a.split_den, n, v)) continue;
        }
        const int64_t nrows = (int64_t)K + (c1 - c0);
        if (PASS == 1 && nrows > kHeavyRows) continue;  // the heavy pass takes it
        // the rows [r_lo, r_hi) this warp takes: all of the hub's, or one item's group
        const int64_t r_lo = heavy ? (int64_t)grp * kItemRows : 0;
        const int64_t r_hi = heavy ? min(nrows, r_lo + kItemRows) : nrows;
        // INC: no arc of the hub is new, so every pair of its tile was met through
        // arcs of G_{r-2}, in the previous round's pool, and none can change G_r
        // (the fast path reads the first 32 flags with the ids)
        // (an item of the heavy pass: its rows and the columns, the hub's first K rows)
        if (INC && !fast) {
            bool any = false;
            for (int64_t r = lane; r < K; r += 32) any |= row_new(a, v, K, c0, r) != 0;
            for (int64_t r = max(r_lo, (int64_t)K) + lane; r < r_hi; r += 32) any |= row_new(a, v, K, c0, r) != 0;
            if (!__any_sync(0xffffffffu, any)) continue;
        }
        // the hub's own log row: column v of the co-friend pairs, row slot 32
        for (int i4 = lane; i4 < MP / 4; i4 += 32)
            reinterpret_cast<float4 *>(sX + 32 * S::RS)[i4] =
                __ldg(reinterpret_cast<const float4 *>(a.L32 + v * MP) + i4);
        int rid0 = -1;  // fast: this lane's row of the first chunk
        int rnew0 = 1;
        if (fast) {
            if (lane < nrows) {
                rid0 = lane < K ? a.idx[v * K + lane] : a.cof[c0 + (lane - K)];
                if (INC) rnew0 = row_new(a, v, K, c0, lane);
                if (!valid_id(rid0, n)) {
                    atomicOr(a.err, kErrIndex);
                    rid0 = -1;
                }
            }
            if (INC) {
                bool any = lane < nrows && rnew0;
                for (int64_t r = 32 + lane; r < nrows; r += 32) any |= row_new(a, v, K, c0, r) != 0;
                if (!__any_sync(0xffffffffu, any)) continue;
            }
            if (lane < K) {
                sCid[lane] = rid0;
                if (INC) sCnew[lane] = (unsigned char)rnew0;
                if (COL) sH[lane] = rid0 >= 0 ? __double2float_rd(a.negH[rid0] * a.col_inv) : 0.f;
            }
        } else {
            for (int j = lane; j < K; j += 32) {
                int id = a.idx[v * K + j];
                if (!valid_id(id, n)) {
                    atomicOr(a.err, kErrIndex);
                    id = -1;
                }
                sCid[j] = id;
                if (INC) sCnew[j] = (unsigned char)row_new(a, v, K, c0, j);
                if (COL) sH[j] = id >= 0 ? __double2float_rd(a.negH[id] * a.col_inv) : 0.f;
            }
        }
        // COL: the hub's own column value, for the co-friend pairs (y = v)
        const float hv = COL ? __double2float_rd(a.negH[v] * a.col_inv) : 0.f;
        __syncwarp();
        // no new column: only rows reached through a new arc can propose
        const bool any_col_new =
            !INC || __any_sync(0xffffffffu, lane < K && sCnew[lane]) ||
            (K > 32 && __any_sync(0xffffffffu, lane + 32 < K && sCnew[lane + 32]));
        const int idA = (active && cA < K) ? sCid[cA] : -1;
        const int idB = (active && cB < K) ? sCid[cB] : -1;
        // MP = 128: two columns' log rows do not fit in registers; the scoring runs
        // over CHK coordinates at a time, the partial dots carried in the dot buffer
        // (each chunk's two chains start from the partial dot and zero)
        constexpr int CHK = MP <= 96 ? MP : 32;
        constexpr int NCH = MP / CHK;
        float LA[CHK], LB[CHK];
        float ph0 = 0.f;
        int64_t roff0 = 0;
        if (fast) {
            constexpr int Q = MP / 4;
            float4 cv[Q], xv[Q];
#pragma unroll
            for (int t = 0; t < Q; ++t) {
                const int i = lane + 32 * t, j = i / Q, c = i - j * Q;
                const int id = j < K ? sCid[j] : -1;
                cv[t] = id >= 0 ? __ldg(reinterpret_cast<const float4 *>(a.L32 + (int64_t)id * MP) + c)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float4 *xr = reinterpret_cast<const float4 *>(a.X32 + (int64_t)(rid0 < 0 ? 0 : rid0) * MP);
#pragma unroll
            for (int i4 = 0; i4 < Q; ++i4) xv[i4] = rid0 >= 0 ? __ldg(xr + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (rid0 >= 0) {
                const RowMeta rm = a.meta[rid0];
                ph0 = rm.phi;
                roff0 = rm.boff;
            }
            float4 *sC4 = reinterpret_cast<float4 *>(sD);
#pragma unroll
            for (int t = 0; t < Q; ++t) {
                const int i = lane + 32 * t, j = i / Q, c = i - j * Q;
                if (j < K) sC4[j * (CS / 4) + c] = cv[t];
            }
            float4 *srow = reinterpret_cast<float4 *>(sX + lane * S::RS);
#pragma unroll
            for (int i4 = 0; i4 < Q; ++i4) srow[i4] = xv[i4];
            __syncwarp();
            const float4 *ra = sC4 + (idA >= 0 ? cA : 0) * (CS / 4);
            const float4 *rb = sC4 + (idB >= 0 ? cB : 0) * (CS / 4);
#pragma unroll
            for (int i4 = 0; i4 < Q; ++i4) {
                const float4 ta = idA >= 0 ? ra[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 tb = idB >= 0 ? rb[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
                LA[4 * i4 + 0] = ta.x; LA[4 * i4 + 1] = ta.y; LA[4 * i4 + 2] = ta.z; LA[4 * i4 + 3] = ta.w;
                LB[4 * i4 + 0] = tb.x; LB[4 * i4 + 1] = tb.y; LB[4 * i4 + 2] = tb.z; LB[4 * i4 + 3] = tb.w;
            }
            __syncwarp();  // the dot buffer is written by the scoring below
        } else if (NCH == 1) {
            const float4 *ra = reinterpret_cast<const float4 *>(a.L32 + (int64_t)(idA < 0 ? 0 : idA) * MP);
            const float4 *rb = reinterpret_cast<const float4 *>(a.L32 + (int64_t)(idB < 0 ? 0 : idB) * MP);
#pragma unroll
            for (int i4 = 0; i4 < CHK / 4; ++i4) {
                const float4 ta = (idA >= 0) ? __ldg(ra + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 tb = (idB >= 0) ? __ldg(rb + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
                LA[4 * i4 + 0] = ta.x; LA[4 * i4 + 1] = ta.y; LA[4 * i4 + 2] = ta.z; LA[4 * i4 + 3] = ta.w;
                LB[4 * i4 + 0] = tb.x; LB[4 * i4 + 1] = tb.y; LB[4 * i4 + 2] = tb.z; LB[4 * i4 + 3] = tb.w;
            }
        }

        for (int64_t base = r_lo; base < r_hi; base += 32) {
            const int nr = (int)min((int64_t)32, r_hi - base);
            // stage: lane t <-> row t of the chunk
            const int64_t r = base + lane;
            int rid = -1;
            int rnew = 1;
            float ph = 0.f;
            int64_t roff = 0;
            if (fast && base == 0) {  // staged above
                rid = rid0;
                rnew = rnew0;
                ph = ph0;
                roff = roff0;
            } else {
                if (r < r_hi) {  // rows past r_hi belong to the next item
                    rid = (r < K) ? a.idx[v * K + r] : a.cof[c0 + (r - K)];
                    if (INC) rnew = row_new(a, v, K, c0, r);
                    if (!valid_id(rid, n)) {
                        atomicOr(a.err, kErrIndex);
                        rid = -1;
                    }
                }
                float4 *srow = reinterpret_cast<float4 *>(sX + lane * S::RS);
                if (rid >= 0) {
                    const RowMeta rm = a.meta[rid];
                    ph = rm.phi;
                    roff = rm.boff;
                    const float4 *xr = reinterpret_cast<const float4 *>(a.X32 + (int64_t)rid * MP);
#pragma unroll
                    for (int i4 = 0; i4 < MP / 4; ++i4) srow[i4] = __ldg(xr + i4);
                } else {
#pragma unroll
                    for (int i4 = 0; i4 < MP / 4; ++i4) srow[i4] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncwarp();
            }
            // score: group g takes rows it*2G + 2g and +1
            for (int ch = 0; ch < NCH; ++ch) {
                if (NCH > 1) {
                    const float4 *ra = reinterpret_cast<const float4 *>(a.L32 + (int64_t)(idA < 0 ? 0 : idA) * MP) +
                                       ch * (CHK / 4);
                    const float4 *rb = reinterpret_cast<const float4 *>(a.L32 + (int64_t)(idB < 0 ? 0 : idB) * MP) +
                                       ch * (CHK / 4);
#pragma unroll
                    for (int i4 = 0; i4 < CHK / 4; ++i4) {
                        const float4 ta = (idA >= 0) ? __ldg(ra + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 tb = (idB >= 0) ? __ldg(rb + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        LA[4 * i4 + 0] = ta.x; LA[4 * i4 + 1] = ta.y; LA[4 * i4 + 2] = ta.z; LA[4 * i4 + 3] = ta.w;
                        LB[4 * i4 + 0] = tb.x; LB[4 * i4 + 1] = tb.y; LB[4 * i4 + 2] = tb.z; LB[4 * i4 + 3] = tb.w;
                    }
                }
                for (int r0 = 2 * g; r0 < nr; r0 += 2 * G) {
                    if (!active) break;
                    const int r1 = r0 + 1;  // row 32 of sX is the hub row: harmless when r1 == nr
                    const float4 *x0 = reinterpret_cast<const float4 *>(sX + r0 * S::RS) + ch * (CHK / 4);
                    const float4 *x1 = reinterpret_cast<const float4 *>(sX + r1 * S::RS) + ch * (CHK / 4);
                    // each dot as two chains, over the even and the odd coordinates, run
                    // together by packed two-wide fmas and added at the end of the chunk
                    // (the co-friend pair below follows the same order)
                    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
                    if (ch > 0) {  // this lane's own cells of the previous chunk
                        if (cA < K) {
                            a0.x = sD[r0 * DS + cA];
                            if (r1 < nr) a1.x = sD[r1 * DS + cA];
                        }
                        if (cB < K) {
                            b0.x = sD[r0 * DS + cB];
                            if (r1 < nr) b1.x = sD[r1 * DS + cB];
                        }
                    }
#pragma unroll
                    for (int i4 = 0; i4 < CHK / 4; ++i4) {
                        const float4 u = x0[i4], w = x1[i4];
                        const float2 la0 = make_float2(LA[4 * i4 + 0], LA[4 * i4 + 1]);
                        const float2 la1 = make_float2(LA[4 * i4 + 2], LA[4 * i4 + 3]);
                        const float2 lb0 = make_float2(LB[4 * i4 + 0], LB[4 * i4 + 1]);
                        const float2 lb1 = make_float2(LB[4 * i4 + 2], LB[4 * i4 + 3]);
                        a0 = __ffma2_rn(make_float2(u.x, u.y), la0, a0);
                        a1 = __ffma2_rn(make_float2(w.x, w.y), la0, a1);
                        b0 = __ffma2_rn(make_float2(u.x, u.y), lb0, b0);
                        b1 = __ffma2_rn(make_float2(w.x, w.y), lb0, b1);
                        a0 = __ffma2_rn(make_float2(u.z, u.w), la1, a0);
                        a1 = __ffma2_rn(make_float2(w.z, w.w), la1, a1);
                        b0 = __ffma2_rn(make_float2(u.z, u.w), lb1, b0);
                        b1 = __ffma2_rn(make_float2(w.z, w.w), lb1, b1);
                    }
                    if (cA < K) {
                        sD[r0 * DS + cA] = __fadd_rn(a0.x, a0.y);
                        if (r1 < nr) sD[r1 * DS + cA] = __fadd_rn(a1.x, a1.y);
                    }
                    if (cB < K) {
                        sD[r0 * DS + cB] = __fadd_rn(b0.x, b0.y);
                        if (r1 < nr) sD[r1 * DS + cB] = __fadd_rn(b1.x, b1.y);
                    }
                }
            }
            __syncwarp();
            // filter: lane t <-> row t; survivors compacted in place in the row's dots,
            // their column numbers in sJ
            int q = 0;
            if (lane < nr && rid >= 0 && (!INC || rnew || any_col_new)) {
                float *drow = sD + lane * DS;
                unsigned char *jrow = sJ + lane * K;
                for (int j = 0; j < K; ++j) {
                    const float d = drow[j];
                    const int cj = sCid[j];
                    const float thr = COL ? __fsub_rd(sH[j], ph) : ph;
                    if (cj >= 0 && cj != rid && d >= thr && (!INC || rnew || sCnew[j])) {
                        drow[q] = d;
                        jrow[q] = (unsigned char)j;
                        ++q;
                    }
                }
            }
            // co-friend pair (x in F(v), y = v)
            bool cfpass = false;
            float cfd = 0.f;
            if (r < K && rid >= 0 && (!INC || rnew)) {
                const float4 *xr = reinterpret_cast<const float4 *>(sX + lane * S::RS);
                const float4 *lv = reinterpret_cast<const float4 *>(sX + 32 * S::RS);
                // the scoring's order (chunks of CHK, two chains each): the same pair met
                // at another hub as row and column gets the same FP32 value, so that the
                // merge recognises the copies of one candidate
                float acc = 0.f;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    float2 e = make_float2(acc, 0.f);
#pragma unroll
                    for (int i4 = ch * (CHK / 4); i4 < (ch + 1) * (CHK / 4); ++i4) {
                        const float4 xv = xr[i4], lw = lv[i4];
                        e = __ffma2_rn(make_float2(xv.x, xv.y), make_float2(lw.x, lw.y), e);
                        e = __ffma2_rn(make_float2(xv.z, xv.w), make_float2(lw.z, lw.w), e);
                    }
                    acc = __fadd_rn(e.x, e.y);
                }
                cfd = acc;
                cfpass = acc >= (COL ? __fsub_rd(hv, ph) : ph);
            }
            const int count = q + (cfpass ? 1 : 0);
            int64_t rowbase = -1;
            if (count > 0) {
                const int p = atomicAdd(&a.bcnt[rid], count);
                rowbase = roff + p;
                if (a.debug) {
                    const int64_t cap = (int64_t)K * K + (int64_t)(K + 1) * (a.cof_off[rid + 1] - a.cof_off[rid]);
                    if (p + count > cap) {
                        atomicOr(a.err, kErrBucket);
                        rowbase = -1;
                    }
                }
                if (cfpass && rowbase >= 0)
                    a.bent[rowbase + q] =
                        make_int2((int)sortable_bits(COL ? __fmul_rn(a.col_scale, __fsub_rn(hv, cfd)) : -cfd),
                                  (int)v);
            }
            // coalesced writes of the column survivors: entry k of the chunk's
            // flattened list goes to row t = the first with prefix > k
            int incl = q;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
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
                const int t = lo;
                const int qq = k - (t ? sInc[t - 1] : 0);
                const int64_t rb = sRB[t];
                if (rb >= 0) {
                    const int j = sJ[t * K + qq];
                    const float d = sD[t * DS + qq];
                    // the entry orders the candidates like their keys: -d, or s (co(y)/s - d)
                    a.bent[rb + qq] = make_int2(
                        (int)sortable_bits(COL ? __fmul_rn(a.col_scale, __fsub_rn(sH[j], d)) : -d), sCid[j]);
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ FP64
template <int MP, int CPL>
struct F64Smem {
    static constexpr int RS = MP + 2;  // row stride in doubles (16-byte aligned)
    static constexpr int X_DOUBLES = 33 * RS;
    static constexpr int D_DOUBLES = CPL * 32 * 33;
    static constexpr int WARP_DOUBLES = X_DOUBLES + D_DOUBLES;
};

template <int MP, int CPL>
__global__ void __launch_bounds__(128) join_fp64_kernel(JoinArgs a)
{
    using S = F64Smem<MP, CPL>;
    extern __shared__ double2 smemd[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double *sX = reinterpret_cast<double *>(smemd) + warp * S::WARP_DOUBLES;
    double *sD = sX + S::X_DOUBLES;
    const int K = a.K;
    const int64_t n = a.n;
    const unsigned FULL = 0xffffffffu;

    for (int64_t v = a.h_lo + (int64_t)blockIdx.x * wpb + warp; v < a.h_hi; v += (int64_t)gridDim.x * wpb) {
        if (!a.iv.live(v)) continue;  // hub of a stopped instance (batched form)
        if (!in_phase(a.iv, a.phase, a.split_den, n, v)) continue;
        if (a.flag) {  // incremental proposals: a hub with no new arc has nothing to propose
            const int64_t h0 = a.cof_off[v], hn = (int64_t)K + (a.cof_off[v + 1] - h0);
            bool any = false;
            for (int64_t r = lane; r < hn; r += 32) any |= row_new(a, v, K, h0, r) != 0;
            if (!__any_sync(FULL, any)) continue;
        }
        int cid[CPL], cnew[CPL];
        double cnh[CPL];  // column offsets (reverse KL: negH(y); squared Euclidean: |y|^2)
        double Lc[CPL][MP];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int j = lane + 32 * c;
            int id = -1;
            cnew[c] = 0;
            if (j < K) {
                id = a.idx[v * K + j];
                cnew[c] = row_new(a, v, K, 0, j);
                if (!valid_id(id, n)) {
                    atomicOr(a.err, kErrIndex);
                    id = -1;
                }
            }
            cid[c] = id;
            cnh[c] = (has_col_offset(a.cmp) && id >= 0) ? a.negH[id] : 0.0;
            const double2 *lr = reinterpret_cast<const double2 *>(a.L64 + (int64_t)(id < 0 ? 0 : id) * MP);
#pragma unroll
            for (int i2 = 0; i2 < MP / 2; ++i2) {
                double2 t = (id >= 0) ? __ldg(lr + i2) : make_double2(0.0, 0.0);
                Lc[c][2 * i2 + 0] = t.x;
                Lc[c][2 * i2 + 1] = t.y;
            }
        }
        for (int i2 = lane; i2 < MP / 2; i2 += 32)
            reinterpret_cast<double2 *>(sX + 32 * S::RS)[i2] =
                __ldg(reinterpret_cast<const double2 *>(a.L64 + v * MP) + i2);

        const int64_t c0 = a.cof_off[v];
        const int64_t nrows = (int64_t)K + (a.cof_off[v + 1] - c0);
        for (int64_t base = 0; base < nrows; base += 32) {
            const int nr = (int)min((int64_t)32, nrows - base);
            const int64_t r = base + lane;
            int rid = -1, rnew = 1;
            if (r < nrows) {
                rid = (r < K) ? a.idx[v * K + r] : a.cof[c0 + (r - K)];
                rnew = row_new(a, v, K, c0, r);
                if (!valid_id(rid, n)) {
                    atomicOr(a.err, kErrIndex);
                    rid = -1;
                }
            }
            double nh = 0.0, tk = 0.0;
            int ik = 0;
            int64_t roff = 0;
            double2 *srow = reinterpret_cast<double2 *>(sX + lane * S::RS);
            if (rid >= 0) {
                nh = a.negH[rid];
                tk = a.tau[rid];
                ik = a.idxK[rid];
                roff = (int64_t)K * K * rid + (int64_t)(K + 1) * a.cof_off[rid];
                const double2 *xr = reinterpret_cast<const double2 *>(a.X64 + (int64_t)rid * MP);
#pragma unroll
                for (int i2 = 0; i2 < MP / 2; ++i2) srow[i2] = __ldg(xr + i2);
            } else {
#pragma unroll
                for (int i2 = 0; i2 < MP / 2; ++i2) srow[i2] = make_double2(0.0, 0.0);
            }
            __syncwarp();

            unsigned mymask[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) mymask[c] = 0u;
            for (int rr = 0; rr < nr; ++rr) {
                const int rrid = __shfl_sync(FULL, rid, rr);
                const double rnh = __shfl_sync(FULL, nh, rr);
                const double rtk = __shfl_sync(FULL, tk, rr);
                const int rik = __shfl_sync(FULL, ik, rr);
                const int rrnew = __shfl_sync(FULL, rnew, rr);
                const double2 *xr = reinterpret_cast<const double2 *>(sX + rr * S::RS);
                double acc[CPL];
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = 0.0;
#pragma unroll
                for (int i2 = 0; i2 < MP / 2; ++i2) {
                    const double2 xv = xr[i2];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        acc[c] = __fma_rn(xv.x, Lc[c][2 * i2 + 0], acc[c]);
                        acc[c] = __fma_rn(xv.y, Lc[c][2 * i2 + 1], acc[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const double k = !has_col_offset(a.cmp)         ? rnh - acc[c]
                                     : a.cmp == KNND_CMP_KL_REVERSE ? cnh[c] - acc[c]
                                                                    : (rnh - 2.0 * acc[c]) + cnh[c];
                    const bool pass = rrid >= 0 && cid[c] >= 0 && cid[c] != rrid && (rrnew || cnew[c]) &&
                                      lex_less(k, cid[c], rtk, rik);
                    const unsigned m = __ballot_sync(FULL, pass);
                    if (lane == rr) mymask[c] = m;
                    sD[(c * 32 + rr) * 33 + lane] = k;
                }
            }
            bool cfpass = false;
            double cfk = 0.0;
            if (r < K && rid >= 0) {
                const double2 *xr = reinterpret_cast<const double2 *>(sX + lane * S::RS);
                const double2 *lv = reinterpret_cast<const double2 *>(sX + 32 * S::RS);
                double acc = 0.0;
#pragma unroll
                for (int i2 = 0; i2 < MP / 2; ++i2) {
                    const double2 xv = xr[i2], lw = lv[i2];
                    acc = __fma_rn(xv.x, lw.x, acc);
                    acc = __fma_rn(xv.y, lw.y, acc);
                }
                cfk = !has_col_offset(a.cmp)         ? nh - acc
                      : a.cmp == KNND_CMP_KL_REVERSE ? a.negH[v] - acc
                                                     : (nh - 2.0 * acc) + a.negH[v];
                cfpass = rnew && lex_less(cfk, (int)v, tk, ik);
            }
            int count = cfpass ? 1 : 0;
#pragma unroll
            for (int c = 0; c < CPL; ++c) count += __popc(mymask[c]);
            int64_t rowbase = 0;
            if (count > 0) {
                const int p = atomicAdd(&a.bcnt[rid], count);
                rowbase = roff + p;
                if (a.debug) {
                    const int64_t cap = (int64_t)K * K + (int64_t)(K + 1) * (a.cof_off[rid + 1] - a.cof_off[rid]);
                    if (p + count > cap) {
                        atomicOr(a.err, kErrBucket);
                        count = 0;
                        cfpass = false;
                        rowbase = -1;
                    }
                }
            }
            const unsigned lt = lanemask_lt();
            for (int rr = 0; rr < nr; ++rr) {
                int64_t rb = __shfl_sync(FULL, rowbase, rr);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const unsigned m = __shfl_sync(FULL, mymask[c], rr);
                    if (rb >= 0 && ((m >> lane) & 1u)) {
                        const int64_t pos = rb + __popc(m & lt);
                        const double k = sD[(c * 32 + rr) * 33 + lane];
                        a.bkey[pos] = k;
                        a.bent[pos] = make_int2((int)sortable_bits(__double2float_ru(k)), cid[c]);
                    }
                    rb += __popc(m);
                }
            }
            if (cfpass && rowbase >= 0) {
                a.bkey[rowbase + count - 1] = cfk;
                a.bent[rowbase + count - 1] = make_int2((int)sortable_bits(__double2float_ru(cfk)), (int)v);
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ dispatch
template <int MP, int CPL>
static cudaError_t run_join(knnd_handle *h, const JoinArgs &a)
{
    if (h->prec == KNND_PREC_FP64) {
        using S = F64Smem<MP, CPL>;
        const int threads = 128;
        const size_t smem = sizeof(double) * S::WARP_DOUBLES * (threads / 32);
        cudaFuncSetAttribute(join_fp64_kernel<MP, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, join_fp64_kernel<MP, CPL>, threads, smem);
        if (per_sm < 1) per_sm = 1;
        const int64_t need = (a.h_hi - a.h_lo + threads / 32 - 1) / (threads / 32);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)h->num_sms * per_sm));
        join_fp64_kernel<MP, CPL><<<(unsigned)grid, threads, smem, h->stream>>>(a);
    } else {
        using S = MixedSmem<MP>;
        const int threads = 128;
        const size_t smem = (size_t)S::warp_bytes(h->K) * (threads / 32);
        const bool col = has_col_offset(a.cmp);
        // the heavy pass runs for the inner product, whose graphs are hub-heavy (the
        // points of largest norm become nearly everyone's friend); the divergences'
        // and the distance's in-degrees stay near K, where it would add two launches
        // per join for nothing.  Incremental proposals keep one pass.
        const bool split_heavy = !a.flag && a.cmp == KNND_CMP_INNER;
        auto kern = split_heavy ? join_mixed_kernel<MP, false, false, 1>
                    : col ? (a.flag ? join_mixed_kernel<MP, true, true, 0> : join_mixed_kernel<MP, false, true, 0>)
                          : (a.flag ? join_mixed_kernel<MP, true, false, 0> : join_mixed_kernel<MP, false, false, 0>);
        auto hkern = join_mixed_kernel<MP, false, false, 2>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(hkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (per_sm < 1) per_sm = 1;
        const int64_t need = (a.h_hi - a.h_lo + threads / 32 - 1) / (threads / 32);
        const int64_t full = (int64_t)h->num_sms * per_sm;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, full));
        JoinArgs m = a;
        m.items = split_heavy ? h->heavy_items : nullptr;
        m.nitems = h->heavy_nitems;
        m.heavy_pass = 0;
        if (m.items) {  // the heavy hubs' items, then the main pass, then the items
            cudaMemsetAsync(h->heavy_nitems, 0, sizeof(int32_t), h->stream);
            const int64_t hub_blocks = (a.h_hi - a.h_lo + 255) / 256;
            heavy_items_kernel<<<(unsigned)std::max<int64_t>(1, hub_blocks), 256, 0, h->stream>>>(m, h->heavy_items,
                                                                                             h->heavy_nitems);
        }
        kern<<<(unsigned)grid, threads, smem, h->stream>>>(m);
        if (m.items) {
            m.heavy_pass = 1;
            hkern<<<(unsigned)full, threads, smem, h->stream>>>(m);
        }
    }
    return cudaGetLastError();
}

template <int MP>
static cudaError_t run_join_cpl(knnd_handle *h, const JoinArgs &a)
{
    if (h->K <= 32) return run_join<MP, 1>(h, a);
    return run_join<MP, 2>(h, a);
}

static bool join_runs_tc(const knnd_handle *h)
{
    return h->prec == KNND_PREC_MIXED_BF16X3 && tc_supported(h->MP, h->K) && h->prm.comparator == KNND_CMP_KL;
}

bool join_runs_tma(const knnd_handle *h)
{
    return !join_runs_tc(h) && h->join_form == KNND_JOIN_TMA && tma_join_supported(h);
}

cudaError_t launch_join(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase, int split_den)
{
    if (join_runs_tc(h)) {
        h->join_kernel = KNND_JOIN_TC;
        return launch_join_tc(h, idx, h_lo, h_hi, phase, split_den);
    }
    if (join_runs_tma(h)) {
        cudaMemsetAsync(h->bcnt, 0, sizeof(int32_t) * h->n, h->stream);
        h->launches += 1;
        h->join_kernel = KNND_JOIN_TMA;
        return launch_join_tma(h, idx, h_lo, h_hi, phase, split_den);
    }
    h->join_kernel = h->prec == KNND_PREC_FP64 ? KNND_JOIN_FP64 : KNND_JOIN_PLAIN;
    JoinArgs a;
    a.n = h->n;
    a.h_lo = h_lo;
    a.h_hi = h_hi;
    a.phase = phase;
    a.split_den = split_den;
    a.items = nullptr;
    a.nitems = nullptr;
    a.heavy_pass = 0;
    a.K = h->K;
    a.idx = idx;
    a.cof_off = h->cof_off;
    a.cof = h->cof;
    a.X32 = h->X32;
    a.L32 = h->L32;
    a.X64 = h->X64;
    a.L64 = h->L64;
    a.negH = h->negH;
    a.tau = h->tau;
    a.idxK = h->idxK;
    a.meta = h->meta;
    a.bcnt = h->bcnt;
    a.bent = h->bent;
    a.bkey = h->bkey;
    a.err = h->err;
    a.debug = h->prm.debug;
    a.iv = h->iv;
    a.flag = h->round_flag;
    a.cof_new = h->round_flag ? h->cof_new : nullptr;
    a.cmp = h->prm.comparator;
    a.col_scale = a.cmp == KNND_CMP_SQEUCLIDEAN ? 2.f : 1.f;
    a.col_inv = a.cmp == KNND_CMP_SQEUCLIDEAN ? 0.5 : 1.0;
    if (a.cmp == KNND_CMP_KL_REVERSE) {  // rows read log x, columns read y
        std::swap(a.X32, a.L32);
        std::swap(a.X64, a.L64);
    }
    cudaMemsetAsync(h->bcnt, 0, sizeof(int32_t) * h->n, h->stream);
    h->launches += 1;
    switch (h->MP) {
    case 8: return run_join_cpl<8>(h, a);
    case 16: return run_join_cpl<16>(h, a);
    case 24: return run_join_cpl<24>(h, a);
    case 32: return run_join_cpl<32>(h, a);
    case 48: return run_join_cpl<48>(h, a);
    case 64: return run_join_cpl<64>(h, a);
    case 72: return run_join_cpl<72>(h, a);
    case 96: return run_join_cpl<96>(h, a);
    case 128: return run_join_cpl<128>(h, a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace knnd
