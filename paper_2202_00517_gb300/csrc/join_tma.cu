// join_tma.cu -- the FP32 filter of the local join (Sec. 3.1 "Meet", Sec. 4.2)
// with its rows and columns brought into shared memory by the TMA engine.
//
// Same hub tiles, filter, bucket entries and error bound as join_mixed_kernel
// (join.cu): hub v's rows are F(v) then coF(v), its columns F(v) and, for the
// rows of F(v), v itself; a pair is kept when its FP32 dot can still beat the
// row's K-th entry.  Here the co-friends that are also friends of v are left
// out of the rows (their pairs are those of their first row; launch_reverse_csr
// places them last in each list).  What differs besides is how the tile reaches the FP32
// pipe:
//
//  * a warp takes a hub's rows 32 R at a time (an item; R = 1 is the one
//    instantiated); lane t owns row t of the item (and t + 32 when R = 2) for
//    the whole item: its coordinates sit in registers, so the dots of a row are
//    finished in the lane that filters them and never pass through shared
//    memory;
//  * the 32 rows of an item and the K + 1 columns of a hub are gathered from
//    the FP32 tables by cp.async.bulk.tensor ... tile::gather4 (four indexed
//    rows of a two-dimensional tensor map per instruction, one row high), which
//    moves them into shared memory without passing through the load/store
//    pipe; an index outside the table (an empty row slot) reads zeros;
//  * the kernel is persistent (as many blocks as fit on the SMs); its warps take
//    hubs from a device work queue, chunks of consecutive hubs claimed by an
//    atomic counter, so the load spreads by what each hub costs;
//  * the copies of the next item are issued as soon as the current item's rows
//    have left the staging buffer, and the ids of the item after it are loaded
//    while the current item is scored, so gathers, id chases and scoring of
//    three consecutive items overlap within one warp;
//  * every lane reads each column coordinate from shared memory as a broadcast
//    (all lanes, one address) and uses it in one fma of its own row.
//
// Each dot is two fma chains, one over the even and one over the odd
// coordinates, run together by packed two-wide FP32 fmas (__ffma2_rn, one
// instruction for both), then added: at most ceil(m/2) + 1 roundings on any
// term, within the m + 6 that the filter's bound c_m = (m + 6) 2^-24 (1.01)
// allows for (Higham, Sec. 3.1: the bound holds for any summation order).
// debug = 1 audits every dot against FP64 for the comparators whose bound is
// E_x itself.  Incremental proposals and the inner product's heavy-hub pass
// stay with join.cu, and so do the shapes the tuning table gives to it.
//
// Every mbarrier wait is bounded (1 s of the global timer); on a timeout the
// warp sets kErrTimeout, waits (bounded) for its copies in flight and stops.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "knnd_internal.cuh"

namespace knnd {

struct TmaJoinArgs {
    CUtensorMap tm_row;  // the rows' FP32 table (X32; reverse KL: L32), n x MP, box MP x 1
    CUtensorMap tm_col;  // the columns' FP32 table (L32; reverse KL: X32)
    int64_t n;
    int64_t h_lo, h_hi;  // hubs [h_lo, h_hi) of phase `phase` (in_phase)
    int phase, split_den;
    int K, MP;
    const int32_t *idx;
    const int64_t *cof_off;
    const int32_t *ncof;  // per hub: the co-friends that are no friends, at the front of its list
    const int32_t *cof;
    const RowMeta *meta;
    const double *negH;  // column offsets (comparators with one)
    int32_t *bcnt;
    int2 *bent;
    int32_t *err;
    int debug;
    InstView iv;
    unsigned long long *queue;  // the work queue's counter: hubs claimed so far (zeroed per launch)
    float col_scale;
    double col_inv;
    // bound audit (debug, comparators without a column offset): the FP64
    // tables, the bound of each row and the counters it adds to
    const double *X64;
    const double *L64;
    const double *Ex;
    int64_t *cnt;
};

namespace {

constexpr unsigned long long kTmaWaitNs = 1000000000ull;  // 1 s
constexpr int kSlot = 36;  // column ids per slot: K + 1 <= 33, padded

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Polls phase `parity` of the mbarrier until it completes (true) or `limit` ns pass (false).
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, unsigned long long limit)
{
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (it == 0) t0 = now_ns();
        else if ((it & 31) == 0 && now_ns() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void expect_bytes(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Four rows r0..r3 (all MP coordinates) of the tensor map's table -> 4 x MP
// floats at dst; an out-of-range row index reads zeros.
__device__ __forceinline__ void gather4(uint32_t dst, const CUtensorMap *tm, int r0, int r1, int r2, int r3,
                                        uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(tm), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}

// Per-warp shared memory (bytes).  KC: column rows staged, K + 1 rounded up to 4;
// column ids (and, with a column offset, RD(co(y)/s)) in two slots of 36.
struct TmaLayout {
    int MP, K, KC, SVS, NR;
    int off_row, off_col0, off_col1, off_sv, off_cid, off_h, off_inc, off_q0, off_rb, off_mask, off_bar, bytes;
    // R: rows per lane (an item has 32 R rows)
    __host__ __device__ TmaLayout(int mp, int k, bool col, int R) : MP(mp), K(k)
    {
        NR = 32 * R;
        KC = (K + 1 + 3) & ~3;
        SVS = K + 1;                          // survivor slots of a row
        const int rowb = NR * MP * 4;         // a multiple of 128 (MP a multiple of 8)
        const int colb = (KC * MP * 4 + 127) & ~127;
        off_row = 0;
        off_col0 = off_row + rowb;
        off_col1 = off_col0 + colb;
        off_sv = off_col1 + colb;
        off_cid = off_sv + ((NR * SVS * 4 + 15) & ~15);
        off_h = off_cid + 2 * kSlot * 4;
        off_inc = off_h + (col ? 2 * kSlot * 4 : 0);
        off_q0 = off_inc + 32 * 4;
        off_rb = off_q0 + (R > 1 ? 32 * 4 : 0);
        off_mask = off_rb + NR * 8;
        off_bar = off_mask + NR * 4;
        bytes = (off_bar + 3 * 8 + 127) & ~127;
    }
};

// The warp's current position in its hubs: hub v, its item `ch` (rows
// 32 ch .. 32 ch + 31), the start of coF(v) and the hub's row count.
struct Item {
    int64_t v;
    int64_t c0;
    int nrows;
    int ch;
    bool valid;
};

// The warp's walk over the hubs it takes from the launch's work queue: chunks
// of kChunk consecutive hubs of [h_lo, h_hi), each claimed by one atomicAdd on
// the queue counter as the warp reaches it, so warps that meet cheap hubs take
// more of them.  `next` is the next hub to consider; its co-friend offsets are
// loaded one hub ahead of their use.  8 hubs a claim: 2.80 against 2.89 ms per
// launch with 32 at n = 1e6, d = 20, K = 20 (a claim is ~70 us of one warp's work
// there, so the last claims of a launch end closer together); 4 measured the same.
constexpr int kChunk = 8;

struct HubWalk {
    int64_t next, end;  // the claimed chunk [next, end)
    int64_t c0, c1;     // cof_off[next], and the end of its co-friends that are no friends (when next < h_hi)
};

// Called by all lanes of the warp together.
__device__ __forceinline__ void walk_claim(const TmaJoinArgs &a, HubWalk &w)
{
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(a.queue, (unsigned long long)kChunk);
    t = __shfl_sync(0xffffffffu, t, 0);
    w.next = a.h_lo + (int64_t)t;
    w.end = min(w.next + kChunk, a.h_hi);
}

__device__ __forceinline__ void walk_load(const TmaJoinArgs &a, HubWalk &w)
{
    if (w.next < a.h_hi) {
        w.c0 = a.cof_off[w.next];
        w.c1 = w.c0 + a.ncof[w.next];
    }
}

__device__ __forceinline__ void walk_step(const TmaJoinArgs &a, HubWalk &w)
{
    w.next += 1;
    if (w.next >= w.end) walk_claim(a, w);
    walk_load(a, w);
}

// The item after `it`: the hub's next 32 rows, or the first rows of the
// warp's next hub that is live and in the launch's phase.
__device__ __forceinline__ Item next_item(const TmaJoinArgs &a, Item it, HubWalk &w, int span)
{
    if (it.valid && (it.ch + 1) * span < it.nrows) {
        it.ch += 1;
        return it;
    }
    Item r;
    r.valid = false;
    r.v = r.c0 = 0;
    r.nrows = r.ch = 0;
    while (w.next < a.h_hi) {
        const int64_t v = w.next;
        if (!a.iv.live(v) || !in_phase(a.iv, a.phase, a.split_den, a.n, v)) {
            walk_step(a, w);
            continue;
        }
        r.v = v;
        r.c0 = w.c0;
        r.nrows = a.K + (int)(w.c1 - w.c0);
        r.valid = true;
        walk_step(a, w);  // the next hub's offsets in flight until the warp reaches it
        break;
    }
    return r;
}

// Bound audit (debug): the FP32 dot d of row x and column y against the FP64
// dot of the same tables; a difference above the row's bound E_x counts as a
// violation (the filter relies on there being none).
__device__ __noinline__ void audit_pair(const TmaJoinArgs &a, int x, int y, float d, long long &ndot,
                                        long long &nviol)
{
    const int MP = a.MP;
    const double *xr = a.X64 + (int64_t)x * MP;
    const double *lr = a.L64 + (int64_t)y * MP;
    double acc = 0.0;
    for (int i = 0; i < MP; ++i) acc = __fma_rn(xr[i], lr[i], acc);
    ndot += 1;
    if (fabs((double)d - acc) > a.Ex[x]) nviol += 1;
}

// Row `t` (0 <= t < span) of item `it` as stored (-1: no row).  Not yet
// checked, so that the load stays in flight until check_id.
__device__ __forceinline__ int load_id(const TmaJoinArgs &a, const Item &it, int t, int span)
{
    if (!it.valid) return -1;
    const int r = it.ch * span + t;
    if (r >= it.nrows) return -1;
    return r < a.K ? a.idx[it.v * a.K + r] : a.cof[it.c0 + (r - a.K)];
}

// An index outside [0, n) is recorded in the error word and skipped (-1).
__device__ __forceinline__ int check_id(const TmaJoinArgs &a, int id, bool present)
{
    if (present && (id < 0 || (int64_t)id >= a.n)) {
        atomicOr(a.err, kErrIndex);
        return -1;
    }
    return present ? id : -1;
}

__device__ __forceinline__ bool has_row(const Item &it, int t, int span)
{
    return it.valid && it.ch * span + t < it.nrows;
}

}  // namespace

// AUDIT: the debug form (debug = 1) of a comparator without a column offset,
// compiled apart so that the default form carries none of its state.
// R: rows per lane; an item is 32 R rows of a hub, lane t holding rows t and
// (R = 2) t + 32, so that each column coordinate read from shared memory feeds
// R rows' fmas.
template <int MP, bool COL, bool AUDIT, int R>
__global__ void __launch_bounds__(128, R == 2 ? 3 : (MP <= 24 ? 5 : 4))
    join_tma_kernel(const __grid_constant__ TmaJoinArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_tma[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = a.K;
    constexpr int NR = 32 * R;
    const TmaLayout L(MP, K, COL, R);
    long long ndot = 0, nviol = 0;
    unsigned char *wb = smem_tma + (size_t)warp * L.bytes;
    const float *sRow = reinterpret_cast<const float *>(wb + L.off_row);
    float *sSv = reinterpret_cast<float *>(wb + L.off_sv);     // [NR][SVS] survivor dots of each row
    unsigned *sMask = reinterpret_cast<unsigned *>(wb + L.off_mask);  // [NR] columns that passed, per row
    int *sCid = reinterpret_cast<int *>(wb + L.off_cid);       // [2][kSlot] column ids per slot
    float *sH = reinterpret_cast<float *>(wb + L.off_h);        // [2][kSlot] RD(co(y) / s) per slot (COL)
    int *sInc = reinterpret_cast<int *>(wb + L.off_inc);       // [32] inclusive survivor counts of the lanes
    int *sQ0 = reinterpret_cast<int *>(wb + L.off_q0);         // [32] survivors of each lane's first row (R = 2)
    long long *sRB = reinterpret_cast<long long *>(wb + L.off_rb);  // [NR] bucket slot of each row's first survivor
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(wb + L.off_bar);
    const uint32_t row_dst = saddr(wb + L.off_row);
    const uint32_t col_dst0 = saddr(wb + L.off_col0), col_step = (uint32_t)(L.off_col1 - L.off_col0);
    const uint32_t bar_row = saddr(bars), bar_col0 = bar_row + 8u;  // slot s: bar_col0 + 8 s
    const uint32_t row_bytes = (uint32_t)NR * MP * 4u, col_bytes = (uint32_t)L.KC * MP * 4u;
    if (saddr(smem_tma) & 127u) {  // the copies need 128-byte aligned destinations (reported as a failed wait)
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        return;
    }
    if (lane == 0) {
        for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bars + b)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();

    HubWalk walk;
    walk.c0 = walk.c1 = 0;
    walk_claim(a, walk);
    walk_load(a, walk);
    Item none;
    none.valid = false;
    none.v = none.c0 = 0;
    none.nrows = none.ch = 0;

    // Copies of item `it` (lane ids `rid`, row s*32 + lane in rid[s]): its NR rows;
    // with its hub's first item, the hub's columns into column slot `slot` and
    // their ids into sCid (the columns are the hub's first K rows).
    auto issue = [&](const Item &it, const int (&rid)[R], int slot) {
        const bool cols = it.ch == 0;
        if (cols) {
            if (lane < K) sCid[slot * kSlot + lane] = rid[0];
            if (lane == 0) sCid[slot * kSlot + K] = (int)it.v;
            if (COL) {
                if (lane < K)
                    sH[slot * kSlot + lane] = rid[0] >= 0 ? __double2float_rd(a.negH[rid[0]] * a.col_inv) : 0.f;
                if (lane == 0) sH[slot * kSlot + K] = __double2float_rd(a.negH[it.v] * a.col_inv);
            }
        }
        // gather coordinates: lanes 0..8R-1 take rows 4l..4l+3, lanes 8R..8R+KC/4-1
        // the columns 4(l-8R)..4(l-8R)+3
        const int g = lane < 8 * R ? lane : lane - 8 * R;
        int q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * g + i;  // row of the item (lanes < 8R) or column (the others)
            int v = __shfl_sync(FULL, rid[0], r & 31);
            if (R > 1) {
                const int v1 = __shfl_sync(FULL, rid[R - 1], r & 31);
                if (lane < 8 * R && r >= 32) v = v1;
            }
            q[i] = lane < 8 * R ? v : (r < K ? v : (r == K ? (int)it.v : -1));
        }
        __syncwarp();  // every lane's reads of the staging buffer come before the copies below
        if (lane == 0) {
            expect_bytes(bar_row, row_bytes);
            if (cols) expect_bytes(bar_col0 + 8u * slot, col_bytes);
        }
        __syncwarp();
        if (lane < 8 * R) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            gather4(row_dst + (uint32_t)(lane * 4 * MP * 4), &a.tm_row, q[0], q[1], q[2], q[3], bar_row);
        } else if (cols && lane < 8 * R + L.KC / 4) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            gather4(col_dst0 + col_step * slot + (uint32_t)((lane - 8 * R) * 4 * MP * 4), &a.tm_col, q[0], q[1],
                    q[2], q[3], bar_col0 + 8u * slot);
        }
    };

    // prologue: item A's copies in flight, item B's ids loading
    Item A = next_item(a, none, walk, NR);
    if (!A.valid) return;
    int ridA[R], ridB[R];
#pragma unroll
    for (int s = 0; s < R; ++s) ridA[s] = check_id(a, load_id(a, A, s * 32 + lane, NR), has_row(A, s * 32 + lane, NR));
    Item B = next_item(a, A, walk, NR);
#pragma unroll
    for (int s = 0; s < R; ++s) ridB[s] = load_id(a, B, s * 32 + lane, NR);
    int slotA = 0;
    issue(A, ridA, slotA);
    RowMeta mA[R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        mA[s].phi = 0.f;
        mA[s].boff = 0;
        if (ridA[s] >= 0) mA[s] = a.meta[ridA[s]];
    }
    uint32_t prow = 0, pcol = 0;  // phase parities: the row barrier; bit s, column slot s

    while (A.valid) {
        // 1. item A's rows: wait, then this lane's rows into registers
        if (!wait_phase(bar_row, prow, kTmaWaitNs)) {
            atomicOr(a.err, kErrTimeout);
            wait_phase(bar_row, prow, kTmaWaitNs);
            if (A.ch == 0) wait_phase(bar_col0 + 8u * slotA, (pcol >> slotA) & 1u, kTmaWaitNs);
            return;
        }
        prow ^= 1u;
        // rows of the item past the first 32 (R = 2): the second row of each lane is scored
        const bool two = R > 1 && A.ch * NR + 32 < A.nrows;
        float2 x[R][MP / 2];  // coordinates (2i, 2i + 1) of this lane's rows
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const float4 *xr = reinterpret_cast<const float4 *>(sRow + (s * 32 + lane) * MP);
#pragma unroll
            for (int i4 = 0; i4 < MP / 4; ++i4) {
                const float4 t = (s == 0 || two) ? xr[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
                x[s][2 * i4 + 0] = make_float2(t.x, t.y);
                x[s][2 * i4 + 1] = make_float2(t.z, t.w);
            }
        }
        __syncwarp();
        // 2. item B's copies (the staging buffer is free again)
        const int slotB = (B.valid && B.ch == 0) ? slotA ^ 1 : slotA;
#pragma unroll
        for (int s = 0; s < R; ++s) ridB[s] = check_id(a, ridB[s], has_row(B, s * 32 + lane, NR));
        if (B.valid) issue(B, ridB, slotB);
        // 3. item C's ids and item B's row records, in flight while A is scored
        const Item C = next_item(a, B, walk, NR);
        int ridC[R];
#pragma unroll
        for (int s = 0; s < R; ++s) ridC[s] = load_id(a, C, s * 32 + lane, NR);
        RowMeta mB[R];
#pragma unroll
        for (int s = 0; s < R; ++s) {
            mB[s].phi = 0.f;
            mB[s].boff = 0;
            if (ridB[s] >= 0) mB[s] = a.meta[ridB[s]];
        }
        // 4. item A's columns (first item of its hub)
        if (A.ch == 0) {
            if (!wait_phase(bar_col0 + 8u * slotA, (pcol >> slotA) & 1u, kTmaWaitNs)) {
                atomicOr(a.err, kErrTimeout);
                wait_phase(bar_col0 + 8u * slotA, (pcol >> slotA) & 1u, kTmaWaitNs);
                if (B.valid) {
                    wait_phase(bar_row, prow, kTmaWaitNs);
                    if (B.ch == 0) wait_phase(bar_col0 + 8u * slotB, (pcol >> slotB) & 1u, kTmaWaitNs);
                }
                return;
            }
            pcol ^= 1u << slotA;
        }
        // 5. score this lane's rows against the hub's columns, filter, compact
        const float4 *Cb = reinterpret_cast<const float4 *>(wb + (slotA ? L.off_col1 : L.off_col0));
        const int *cid = sCid + slotA * kSlot;
        const float *hcol = sH + slotA * kSlot;
        int q[R];
        unsigned mk[R];  // bit j: column j passed
#pragma unroll
        for (int s = 0; s < R; ++s) mk[s] = 0u;
        for (int j0 = 0; j0 < K; j0 += 4) {
            // column j0 + k: chains over the even and the odd coordinates
            float2 e[R][4];
#pragma unroll
            for (int s = 0; s < R; ++s)
#pragma unroll
                for (int k = 0; k < 4; ++k) e[s][k] = make_float2(0.f, 0.f);
            const float4 *c0 = Cb + j0 * (MP / 4);
#pragma unroll
            for (int i4 = 0; i4 < MP / 4; ++i4) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 u = c0[k * (MP / 4) + i4];
#pragma unroll
                    for (int s = 0; s < R; ++s) {
                        if (s > 0 && !two) continue;
                        e[s][k] = __ffma2_rn(x[s][2 * i4], make_float2(u.x, u.y), e[s][k]);
                        e[s][k] = __ffma2_rn(x[s][2 * i4 + 1], make_float2(u.z, u.w), e[s][k]);
                    }
                }
            }
            // the dot goes to the row's slot j whether it passes or not, and the pass
            // bit needs one compare with the row's point (a column that is the row's
            // own point is no pair); columns past K and columns without a point are
            // masked out once, below
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = j0 + k;   // j <= 31 (K <= 32)
                const int cj = cid[j];  // j < K + 3 < 2 kSlot: inside the slot pair
                const float h = COL ? hcol[j] : 0.f;
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    const float d = __fadd_rn(e[s][k].x, e[s][k].y);
                    if (AUDIT && j < K && ridA[s] >= 0 && cj >= 0 && cj != ridA[s])
                        audit_pair(a, ridA[s], cj, d, ndot, nviol);
                    const float thr = COL ? __fsub_rd(h, mA[s].phi) : mA[s].phi;
                    if (j < K) sSv[(s * 32 + lane) * L.SVS + j] = d;
                    mk[s] |= (d >= thr && cj != ridA[s]) ? 1u << j : 0u;
                }
            }
        }
        {
            // columns 0..K-1 that hold a point (the hub's friend list has no gaps but
            // a slot may read -1 at the ends of the index range)
            const unsigned cvalid = __ballot_sync(FULL, lane < K && cid[lane] >= 0);
#pragma unroll
            for (int s = 0; s < R; ++s) {
                mk[s] = ridA[s] >= 0 ? mk[s] & cvalid : 0u;
                q[s] = __popc(mk[s]);
            }
        }
        // the co-friend pair (x in F(v), y = v): column K, rows of F(v) only (the
        // hub's first K rows: lanes < K of the first item's first rows), in the same
        // fma order as the columns above, so that a pair met again at another hub
        // gets the same FP32 value and the merge sees its copies as one candidate
        if (A.ch == 0) {
            const float4 *cv = Cb + K * (MP / 4);
            float2 e = make_float2(0.f, 0.f);
#pragma unroll
            for (int i4 = 0; i4 < MP / 4; ++i4) {
                const float4 u = cv[i4];
                e = __ffma2_rn(x[0][2 * i4], make_float2(u.x, u.y), e);
                e = __ffma2_rn(x[0][2 * i4 + 1], make_float2(u.z, u.w), e);
            }
            const float acc = __fadd_rn(e.x, e.y);
            if (lane < K && ridA[0] >= 0) {
                if (AUDIT) audit_pair(a, ridA[0], (int)A.v, acc, ndot, nviol);
                const float hv = COL ? hcol[K] : 0.f;
                if (acc >= (COL ? __fsub_rd(hv, mA[0].phi) : mA[0].phi)) {
                    sSv[lane * L.SVS + K] = acc;  // the last survivor of the row
                    ++q[0];
                }
            }
        }
        // 6. reserve each row's bucket slots, then write the item's survivors
        //    coalesced: lane t's entries (its first row's, then its second's) follow
        //    those of lanes < t; entry k belongs to the first lane whose inclusive
        //    prefix exceeds k
#pragma unroll
        for (int s = 0; s < R; ++s) {
            long long rowbase = -1;
            if (q[s] > 0) {
                const int p = atomicAdd(&a.bcnt[ridA[s]], q[s]);
                rowbase = mA[s].boff + p;
                if (a.debug) {
                    const int64_t cap =
                        (int64_t)K * K + (int64_t)(K + 1) * (a.cof_off[ridA[s] + 1] - a.cof_off[ridA[s]]);
                    if (p + q[s] > cap) {
                        atomicOr(a.err, kErrBucket);
                        rowbase = -1;
                    }
                }
            }
            sRB[s * 32 + lane] = rowbase;
            sMask[s * 32 + lane] = mk[s];
        }
        int qtot = q[0];
#pragma unroll
        for (int s = 1; s < R; ++s) qtot += q[s];
        int incl = qtot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        sInc[lane] = incl;
        if (R > 1) sQ0[lane] = q[0];
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
            int qq = k - (t ? sInc[t - 1] : 0);
            int rr = t;  // the item's row: lane t's first row, or (past its survivors) its second
            if (R > 1) {
                const int q0 = sQ0[t];
                if (qq >= q0) {
                    qq -= q0;
                    rr = 32 + t;
                }
            }
            const long long rb = sRB[rr];
            if (rb >= 0) {
                // survivor qq of row rr: its qq-th passing column, or (past them) the hub itself
                const unsigned m = sMask[rr];
                const bool colj = qq < __popc(m);
                const int j = colj ? (int)__fns(m, 0, qq + 1) : K;
                const float d = sSv[rr * L.SVS + j];
                const int y = colj ? cid[j] : (int)A.v;
                // the entry orders the candidates like their keys: -d, or s (co(y)/s - d)
                a.bent[rb + qq] =
                    make_int2((int)sortable_bits(COL ? __fmul_rn(a.col_scale, __fsub_rn(hcol[j], d)) : -d), y);
            }
        }
        __syncwarp();
        // 7. advance
        A = B;
        slotA = slotB;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            ridA[s] = ridB[s];
            mA[s] = mB[s];
            ridB[s] = ridC[s];
        }
        B = C;
    }
    if (AUDIT) {
        for (int o = 16; o > 0; o >>= 1) {
            ndot += __shfl_xor_sync(FULL, ndot, o);
            nviol += __shfl_xor_sync(FULL, nviol, o);
        }
        if (lane == 0) {
            atomicAdd((unsigned long long *)&a.cnt[kCntAudited], (unsigned long long)ndot);
            if (nviol) atomicAdd((unsigned long long *)&a.cnt[kCntBoundViol], (unsigned long long)nviol);
        }
    }
}

// ------------------------------------------------------------------ wide rows
// join_wide_kernel: the same filter for 41..72 real coordinates (MP 48, 64 or
// 72; K <= 32).  One row per lane would hold MP coordinates in registers and
// read every column coordinate once for one row.  Here, as in join_mixed_kernel
// (join.cu), lane (g, p) holds the log rows of two columns in registers and
// reads each coordinate of rows 2g + 2Gi and 2g + 2Gi + 1 (G row groups) once
// for both columns: half the shared-memory reads per fma at these
// widths.  What the TMA adds to that layout: an item's 32 rows and a hub's K + 1
// columns reach shared memory by tile::gather4, so the load/store pipe carries
// no gathered sectors, and the next item's copies (its rows; for a new hub also
// its columns) are in flight while the current item's dots are filtered and
// written.  The dots are the same two fma chains (even and odd coordinates,
// added at the end) as every other FP32 join form, the co-friend pair included,
// so that copies of a pair met at several hubs carry one FP32 value.
struct WideLayout {
    int MP, K, KC, DS;
    int off_row, off_col, off_dot, off_cid, off_h, off_inc, off_rb, off_mask, off_bar, bytes;
    __host__ __device__ WideLayout(int mp, int k, bool col) : MP(mp), K(k)
    {
        KC = (K + 1 + 3) & ~3;                 // columns: F(v), then v, padded to whole gather4s
        DS = (K + 1) | 1;                      // dots of a row: K columns, then the co-friend pair
        off_row = 0;                           // [32][MP] the item's rows
        off_col = off_row + 32 * MP * 4;       // [KC][MP] the hub's columns (multiples of 128 bytes)
        off_dot = off_col + KC * MP * 4;       // [32][DS] the item's dots
        off_cid = off_dot + ((32 * DS * 4 + 15) & ~15);
        off_h = off_cid + 2 * kSlot * 4;       // [2][kSlot] column ids; COL: RD(co(y) / s)
        off_inc = off_h + (col ? 2 * kSlot * 4 : 0);
        off_rb = off_inc + 32 * 4;
        off_mask = off_rb + 32 * 8;
        off_bar = off_mask + 32 * 4;
        bytes = (off_bar + 2 * 8 + 127) & ~127;
    }
};

template <int MP, bool COL>
__global__ void __launch_bounds__(128, 2) join_wide_kernel(const __grid_constant__ TmaJoinArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_tma[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = a.K;
    const WideLayout L(MP, K, COL);
    unsigned char *wb = smem_tma + (size_t)warp * L.bytes;
    const float4 *sRow4 = reinterpret_cast<const float4 *>(wb + L.off_row);
    const float4 *sCol4 = reinterpret_cast<const float4 *>(wb + L.off_col);
    float *sD = reinterpret_cast<float *>(wb + L.off_dot);
    int *sCid = reinterpret_cast<int *>(wb + L.off_cid);
    float *sH = reinterpret_cast<float *>(wb + L.off_h);
    int *sInc = reinterpret_cast<int *>(wb + L.off_inc);
    long long *sRB = reinterpret_cast<long long *>(wb + L.off_rb);
    unsigned *sMask = reinterpret_cast<unsigned *>(wb + L.off_mask);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wb + L.off_bar);
    const uint32_t bar_row = saddr(bars), bar_col = bar_row + 8u;
    const uint32_t row_dst = saddr(wb + L.off_row), col_dst = saddr(wb + L.off_col);
    const uint32_t row_bytes = 32u * MP * 4u, col_bytes = (uint32_t)L.KC * MP * 4u;
    if (saddr(smem_tma) & 127u) {  // the copies need 128-byte aligned destinations (reported as a failed wait)
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        return;
    }
    if (lane == 0) {
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bars + b)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();
    // scoring roles: lane (g, p) = columns p and p + npairs of row group g (the
    // columns 288 bytes apart at MP = 72: consecutive columns spread over four bank
    // groups, so that reading them into registers conflicts 4-way, not 8-way)
    const int npairs = (K + 1) >> 1, G = 32 / npairs;
    const int g = lane / npairs, pr = lane - g * npairs;
    const bool active = g < G;
    const int cA = pr, cB = pr + npairs;

    HubWalk walk;
    walk.c0 = walk.c1 = 0;
    walk_claim(a, walk);
    walk_load(a, walk);
    Item none;
    none.valid = false;
    none.v = none.c0 = 0;
    none.nrows = none.ch = 0;

    // Copies of item `it` (this lane's id `rid` is row `lane` of the item): its 32
    // rows; with `cols` (the hub's first item) also the hub's K + 1 columns, the
    // first K rows and then v, with their ids into column-id slot `slot`.
    auto issue = [&](const Item &it, int rid, bool cols, int slot) {
        if (cols) {
            if (lane < K) sCid[slot * kSlot + lane] = rid;
            if (lane == 0) sCid[slot * kSlot + K] = (int)it.v;
            if (COL) {
                if (lane < K) sH[slot * kSlot + lane] = rid >= 0 ? __double2float_rd(a.negH[rid] * a.col_inv) : 0.f;
                if (lane == 0) sH[slot * kSlot + K] = __double2float_rd(a.negH[it.v] * a.col_inv);
            }
        }
        // lanes 0..7 gather rows 4l..4l+3, lanes 8..8+KC/4-1 the columns 4(l-8)..4(l-8)+3
        const int gq = lane < 8 ? lane : lane - 8;
        int q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * gq + i;
            const int v = __shfl_sync(FULL, rid, r & 31);
            q[i] = lane < 8 ? v : (r < K ? v : (r == K ? (int)it.v : -1));
        }
        __syncwarp();  // every lane's reads of the buffers come before the copies below
        if (lane == 0) {
            expect_bytes(bar_row, row_bytes);
            if (cols) expect_bytes(bar_col, col_bytes);
        }
        __syncwarp();
        if (lane < 8) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            gather4(row_dst + (uint32_t)(lane * 4 * MP * 4), &a.tm_row, q[0], q[1], q[2], q[3], bar_row);
        } else if (cols && lane < 8 + L.KC / 4) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            gather4(col_dst + (uint32_t)((lane - 8) * 4 * MP * 4), &a.tm_col, q[0], q[1], q[2], q[3], bar_col);
        }
    };

    Item A = next_item(a, none, walk, 32);
    if (!A.valid) return;
    int ridA = check_id(a, load_id(a, A, lane, 32), has_row(A, lane, 32));
    int slotA = 0;
    issue(A, ridA, true, slotA);  // the first item of a hub
    uint32_t prow = 0, pcol = 0;   // phase parities of the row and the column barrier
    float2 LA[MP / 2], LB[MP / 2];  // log rows of columns cA and cB, coordinates (2i, 2i + 1)
#pragma unroll
    for (int i = 0; i < MP / 2; ++i) LA[i] = LB[i] = make_float2(0.f, 0.f);

    while (A.valid) {
        // the next item's ids and this item's row records, in flight during the scoring
        const Item B = next_item(a, A, walk, 32);
        int ridB = load_id(a, B, lane, 32);
        RowMeta mA;
        mA.phi = 0.f;
        mA.boff = 0;
        if (ridA >= 0) mA = a.meta[ridA];
        const int *cid = sCid + slotA * kSlot;
        const float *hcol = sH + slotA * kSlot;
        // 1. a new hub: its columns into registers
        if (A.ch == 0) {
            if (!wait_phase(bar_col, pcol, kTmaWaitNs)) {
                atomicOr(a.err, kErrTimeout);
                wait_phase(bar_row, prow, kTmaWaitNs);
                return;
            }
            pcol ^= 1u;
            const float4 *ca = sCol4 + (cA < K ? cA : 0) * (MP / 4);
            const float4 *cb = sCol4 + (cB < K ? cB : 0) * (MP / 4);
#pragma unroll
            for (int i4 = 0; i4 < MP / 4; ++i4) {
                const float4 ta = ca[i4], tb = cb[i4];
                LA[2 * i4] = make_float2(ta.x, ta.y);
                LA[2 * i4 + 1] = make_float2(ta.z, ta.w);
                LB[2 * i4] = make_float2(tb.x, tb.y);
                LB[2 * i4 + 1] = make_float2(tb.z, tb.w);
            }
        }
        // 2. the item's rows
        if (!wait_phase(bar_row, prow, kTmaWaitNs)) {
            atomicOr(a.err, kErrTimeout);
            return;
        }
        prow ^= 1u;
        const int nr = min(32, A.nrows - A.ch * 32);
        // 3. dots of rows r0 and r0 + 1 of group g with columns cA and cB: two chains
        //    each, over the even and the odd coordinates, added at the end
        if (active) {
            for (int r0 = 2 * g; r0 < nr; r0 += 2 * G) {
                const int r1 = r0 + 1;  // r0 is even and below 31: row r1 is in the buffer
                const float4 *x0 = sRow4 + r0 * (MP / 4), *x1 = x0 + MP / 4;
                float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
                for (int i4 = 0; i4 < MP / 4; ++i4) {
                    const float4 u = x0[i4], w = x1[i4];
                    a0 = __ffma2_rn(make_float2(u.x, u.y), LA[2 * i4], a0);
                    a1 = __ffma2_rn(make_float2(w.x, w.y), LA[2 * i4], a1);
                    b0 = __ffma2_rn(make_float2(u.x, u.y), LB[2 * i4], b0);
                    b1 = __ffma2_rn(make_float2(w.x, w.y), LB[2 * i4], b1);
                    a0 = __ffma2_rn(make_float2(u.z, u.w), LA[2 * i4 + 1], a0);
                    a1 = __ffma2_rn(make_float2(w.z, w.w), LA[2 * i4 + 1], a1);
                    b0 = __ffma2_rn(make_float2(u.z, u.w), LB[2 * i4 + 1], b0);
                    b1 = __ffma2_rn(make_float2(w.z, w.w), LB[2 * i4 + 1], b1);
                }
                if (cA < K) {
                    sD[r0 * L.DS + cA] = __fadd_rn(a0.x, a0.y);
                    if (r1 < nr) sD[r1 * L.DS + cA] = __fadd_rn(a1.x, a1.y);
                }
                if (cB < K) {
                    sD[r0 * L.DS + cB] = __fadd_rn(b0.x, b0.y);
                    if (r1 < nr) sD[r1 * L.DS + cB] = __fadd_rn(b1.x, b1.y);
                }
            }
        }
        // 4. the co-friend pair (x in F(v), y = v): the rows of F(v), the hub's first
        //    K rows, against column K, in the same order
        float cfd = 0.f;
        const bool cf = A.ch == 0 && lane < K && ridA >= 0;
        if (cf) {
            const float4 *xr = sRow4 + lane * (MP / 4), *cv = sCol4 + K * (MP / 4);
            float2 e = make_float2(0.f, 0.f);
#pragma unroll
            for (int i4 = 0; i4 < MP / 4; ++i4) {
                const float4 xv = xr[i4], lw = cv[i4];
                e = __ffma2_rn(make_float2(xv.x, xv.y), make_float2(lw.x, lw.y), e);
                e = __ffma2_rn(make_float2(xv.z, xv.w), make_float2(lw.z, lw.w), e);
            }
            cfd = __fadd_rn(e.x, e.y);
        }
        __syncwarp();  // the dots are written, the row and column buffers read
        // 5. the next item's copies: the buffers are free (its columns too, if it
        //    starts a hub: this item's columns sit in registers)
        const int slotB = (B.valid && B.ch == 0) ? slotA ^ 1 : slotA;
        ridB = check_id(a, ridB, has_row(B, lane, 32));
        if (B.valid) issue(B, ridB, B.ch == 0, slotB);
        // 6. filter: lane t <-> row t of the item
        unsigned mk = 0u;  // bit j: column j passed
        int q = 0;
        if (ridA >= 0) {  // rows past the item's end have no id
            for (int j = 0; j < K; ++j) {
                const float d = sD[lane * L.DS + j];
                const int cj = cid[j];
                const float thr = COL ? __fsub_rd(hcol[j], mA.phi) : mA.phi;
                mk |= (d >= thr && cj >= 0 && cj != ridA) ? 1u << j : 0u;  // j <= 31
            }
            q = __popc(mk);
            if (cf && cfd >= (COL ? __fsub_rd(hcol[K], mA.phi) : mA.phi)) {
                sD[lane * L.DS + K] = cfd;  // the last survivor of the row
                ++q;
            }
        }
        // 7. reserve each row's bucket slots, then write the item's survivors
        //    coalesced: lane t's entries follow those of lanes < t; entry k belongs
        //    to the first lane whose inclusive prefix exceeds k
        long long rowbase = -1;
        if (q > 0) {
            const int p = atomicAdd(&a.bcnt[ridA], q);
            rowbase = mA.boff + p;
            if (a.debug) {
                const int64_t cap = (int64_t)K * K + (int64_t)(K + 1) * (a.cof_off[ridA + 1] - a.cof_off[ridA]);
                if (p + q > cap) {
                    atomicOr(a.err, kErrBucket);
                    rowbase = -1;
                }
            }
        }
        sRB[lane] = rowbase;
        sMask[lane] = mk;
        int incl = q;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        sInc[lane] = incl;
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
            const long long rb = sRB[t];
            if (rb >= 0) {
                // survivor qq of row t: its qq-th passing column, or (past them) the hub itself
                const unsigned m = sMask[t];
                const bool colj = qq < __popc(m);
                const int j = colj ? (int)__fns(m, 0, qq + 1) : K;
                const float d = sD[t * L.DS + j];
                const int y = colj ? cid[j] : (int)A.v;
                a.bent[rb + qq] =
                    make_int2((int)sortable_bits(COL ? __fmul_rn(a.col_scale, __fsub_rn(hcol[j], d)) : -d), y);
            }
        }
        __syncwarp();
        // 8. advance
        A = B;
        ridA = ridB;
        slotA = slotB;
    }
}

// ------------------------------------------------------------------ host side

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

// A two-dimensional map of an n x MP FP32 table whose box is one whole row
// (the form tile::gather4 takes); rows outside [0, n) read zeros.
bool row_map(CUtensorMap *m, const float *table, int64_t n, int MP)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)MP, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)MP * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)MP, 1u};
    const cuuint32_t es[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(table), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MP, bool COL, int R>
cudaError_t run_tma(knnd_handle *h, const TmaJoinArgs &a)
{
    const int threads = 128;
    const TmaLayout L(MP, h->K, COL, R);
    const size_t smem = (size_t)L.bytes * (threads / 32);
    auto kern = (!COL && a.debug) ? join_tma_kernel<MP, COL, !COL, R> : join_tma_kernel<MP, COL, false, R>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    if (h->join_blocks > 0) per_sm = std::min(per_sm, h->join_blocks);  // the tuned occupancy, if lower
    const int64_t need = (a.h_hi - a.h_lo + threads / 32 - 1) / (threads / 32);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)h->num_sms * per_sm));
    kern<<<(unsigned)grid, threads, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <int MP, bool COL>
cudaError_t run_wide(knnd_handle *h, const TmaJoinArgs &a)
{
    const int threads = 128;
    const WideLayout L(MP, h->K, COL);
    const size_t smem = (size_t)L.bytes * (threads / 32);
    auto kern = join_wide_kernel<MP, COL>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    if (h->join_blocks > 0) per_sm = std::min(per_sm, h->join_blocks);
    const int64_t need = (a.h_hi - a.h_lo + threads / 32 - 1) / (threads / 32);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)h->num_sms * per_sm));
    kern<<<(unsigned)grid, threads, smem, h->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Points below which the tuning table's choice of the TMA join is not followed
// (a caller's explicit knnd_params.join_form is): with fewer hubs than a few per
// resident warp its pipeline never fills (measured: per-instance builds of the
// 4096-instance mix, n <= 50,000, 1.88 s with plain loads against 2.45 s with
// the TMA join).
constexpr int64_t kTmaMinPoints = 65536;

bool tma_join_supported(const knnd_handle *h)
{
    if (h->prm.join_form != KNND_JOIN_TMA && h->n < kTmaMinPoints) return false;
    // MP <= 32: join_tma_kernel; 48..72: join_wide_kernel (no bound audit: debug runs the plain join)
    const bool shape = h->MP <= 32 || ((h->MP == 48 || h->MP == 64 || h->MP == 72) && !h->prm.debug);
    return h->prec != KNND_PREC_FP64 && h->round_flag == nullptr && h->prm.comparator != KNND_CMP_INNER &&
           h->K <= 32 && shape && encode_fn() != nullptr;
}

cudaError_t launch_join_tma(knnd_handle *h, const int32_t *idx, int64_t h_lo, int64_t h_hi, int phase,
                            int split_den)
{
    TmaJoinArgs a;
    std::memset(&a, 0, sizeof(a));
    const int cmp = h->prm.comparator;
    const float *rows = h->X32, *cols = h->L32;
    if (cmp == KNND_CMP_KL_REVERSE) std::swap(rows, cols);  // rows read log x, columns read y
    if (!row_map(&a.tm_row, rows, h->n, h->MP) || !row_map(&a.tm_col, cols, h->n, h->MP))
        return cudaErrorInvalidValue;
    a.n = h->n;
    a.h_lo = h_lo;
    a.h_hi = h_hi;
    a.phase = phase;
    a.split_den = split_den;
    a.K = h->K;
    a.MP = h->MP;
    a.idx = idx;
    a.cof_off = h->cof_off;
    a.ncof = h->deg;  // the front of each coF(v) that launch_reverse_csr kept for this join
    a.cof = h->cof;
    a.meta = h->meta;
    a.negH = h->negH;
    a.bcnt = h->bcnt;
    a.bent = h->bent;
    a.err = h->err;
    a.queue = h->join_queue;
    cudaMemsetAsync(h->join_queue, 0, sizeof(unsigned long long), h->stream);
    a.debug = h->prm.debug;
    a.iv = h->iv;
    a.col_scale = cmp == KNND_CMP_SQEUCLIDEAN ? 2.f : 1.f;
    a.col_inv = cmp == KNND_CMP_SQEUCLIDEAN ? 0.5 : 1.0;
    a.X64 = h->X64;
    a.L64 = h->L64;
    a.Ex = h->Ex;
    a.cnt = h->cnt;
    const bool col = cmp == KNND_CMP_KL_REVERSE || cmp == KNND_CMP_SQEUCLIDEAN;
    // one row per lane: two rows per lane (R = 2: 64-row items, 162 registers, 17.4 KB of shared
    // memory per warp, 12 resident warps per SM) measured 4.05 against 3.10 ms per launch at
    // n = 1e6, d = 20, K = 20, and 3.70 against 2.88 ms with 16 resident warps (the survivor
    // dots kept in the row staging buffer, the next rows gathered after the output)
    switch (h->MP) {
    case 8: return col ? run_tma<8, true, 1>(h, a) : run_tma<8, false, 1>(h, a);
    case 16: return col ? run_tma<16, true, 1>(h, a) : run_tma<16, false, 1>(h, a);
    case 24: return col ? run_tma<24, true, 1>(h, a) : run_tma<24, false, 1>(h, a);
    case 32: return col ? run_tma<32, true, 1>(h, a) : run_tma<32, false, 1>(h, a);
    case 48: return col ? run_wide<48, true>(h, a) : run_wide<48, false>(h, a);
    case 64: return col ? run_wide<64, true>(h, a) : run_wide<64, false>(h, a);
    case 72: return col ? run_wide<72, true>(h, a) : run_wide<72, false>(h, a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace knnd
