// csr.cu -- co-friend lists (Sec. 3.1, Sec. 4.2: "coFriends is derived from
// friends") as a CSR built per round: in-degree count, exclusive scan, fill.
// The count pass also extracts each row's K-th entry, the threshold of the
// join's filter, and (mixed form) the FP32 rejection threshold phi.
#include "knnd_internal.cuh"

namespace knnd {

// Row x's join thresholds from its K-th entry (key t, index v): tau, idxK and,
// mixed form, the FP32 rejection threshold phi and the error bound Ex.
__device__ __forceinline__ void row_thresholds(int64_t x, double t, int32_t v, double *__restrict__ tau,
                                               int32_t *__restrict__ idxK, const double *__restrict__ negH,
                                               const double *__restrict__ nx,
                                               const unsigned long long *__restrict__ smax_bits, const InstView &iv,
                                               double bound_c, int cmp, RowMeta *__restrict__ meta,
                                               double *__restrict__ Ex)
{
    tau[x] = t;
    idxK[x] = v;
    if (meta && (cmp == KNND_CMP_KL || cmp == KNND_CMP_INNER)) {  // inner: negH = 0, L = coordinates
        // |fp32 dot - fp64 dot| <= c_m * sum_i |x_i||log y_i| <= c_m * nx(x) * max|log|.
        // margin covers the FP64 roundings of the key and threshold arithmetic.
        const double smax = __longlong_as_double((long long)smax_bits[3 * iv.at(x)]);
        const double nh = negH[x];
        const double margin = 0x1p-40 * (fabs(nh) + nx[x] * smax + 1.0);
        const double E = bound_c * nx[x] * smax + 0x1p-100 + margin;
        Ex[x] = E;
        meta[x].phi = __double2float_rd(nh - t - E);
    } else if (meta) {
        // comparators with a column offset, key(x, y) = ro(x) - s <R(x), C(y)> + co(y):
        // reverse KL (ro = 0, co = negH(y), s = 1, R = log x, C = y) and squared
        // Euclidean (ro = |x|^2, co = |y|^2, s = 2, R = x, C = y).  The tile's FP32
        // dot d~ is off by at most c_m * sum_i |R_i||C_i| (+ underflow) <=
        // E1 = c_m * max sum_j |y_j| * max |table entry|, per instance.  The join rejects
        // y when d~ < RD(RD(co(y)/s) - phi) with phi = RU((tau - ro)/s + E1 + margin),
        // which proves key > tau.  The candidate's entry is u = s RN(RD(co(y)/s) - d~),
        // and |ro + u - key| <= s E1 + 2^-22 (max|co| + s max sum|y| max|C| + 1) + margin
        // covers the roundings of co/s, of the subtraction and of u: the merge bounds
        // keys by ro + u +- Ex.
        const unsigned long long *mx = smax_bits + 3 * (int64_t)iv.at(x);
        const double smax = __longlong_as_double((long long)mx[0]);
        const double hmax = __longlong_as_double((long long)mx[1]);
        const double nmax = __longlong_as_double((long long)mx[2]);
        const double sc = cmp == KNND_CMP_SQEUCLIDEAN ? 2.0 : 1.0;
        const double ro = cmp == KNND_CMP_SQEUCLIDEAN ? negH[x] : 0.0;
        const double E1 = bound_c * nmax * smax + 0x1p-100;
        const double margin = 0x1p-40 * (fabs(t) + fabs(ro) + hmax + sc * nmax * smax + 1.0);
        Ex[x] = sc * E1 + 0x1p-22 * (hmax + sc * nmax * smax + 1.0) + margin;
        meta[x].phi = __double2float_ru((t - ro) / sc + E1 + margin);
    }
}

// x in F(v)?  f: v's friend list (K entries).
__device__ __forceinline__ bool friend_of(const int32_t *__restrict__ f, int K, int32_t x)
{
    bool hit = false;
    if ((K & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {  // 16-byte aligned rows
        const int4 *f4 = reinterpret_cast<const int4 *>(f);
        for (int q = 0; q < K / 4; ++q) {
            const int4 t = f4[q];
            hit |= (t.x == x) | (t.y == x) | (t.z == x) | (t.w == x);
        }
    } else {
        for (int q = 0; q < K; ++q) hit |= f[q] == x;
    }
    return hit;
}

// One thread per arc e = x*K + t (x -> idx[e]).  With deg_mut (the TMA join's
// rows): a co-friend x of v that is also a friend of v (x in F(v) and v in
// F(x)) stands twice among the hub's rows, F(v) followed by coF(v), and its
// second row proposes exactly the pairs (x, y), y in F(v), of its first; the
// pool of Sec. 3.1 is a set, so the copy adds nothing.  Such arcs are counted
// in deg_mut and placed at the end of coF(v) (slot -1 - k: the k-th from the
// end), the others in deg at its front: the TMA joins read the first deg[v]
// entries, every other consumer the whole list (the same set of pairs).
__global__ void csr_count_kernel(const int32_t *__restrict__ idx, const double *__restrict__ key, int64_t n, int K,
                                 int32_t *__restrict__ deg, int32_t *__restrict__ slot, double *__restrict__ tau,
                                 int32_t *__restrict__ idxK,
                                 const double *__restrict__ negH, const double *__restrict__ nx,
                                 const unsigned long long *__restrict__ smax_bits, InstView iv, double bound_c,
                                 int cmp,
                                 RowMeta *__restrict__ meta, double *__restrict__ Ex, int32_t *err,
                                 int32_t *__restrict__ deg_mut)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int32_t v = idx[e];
    if (v < 0 || v >= n) {
        atomicOr(err, kErrIndex);
    } else if (deg_mut && friend_of(idx + (int64_t)v * K, K, (int32_t)(e / K))) {
        slot[e] = -1 - atomicAdd(&deg_mut[v], 1);  // from the end of coF(v)
    } else {
        slot[e] = atomicAdd(&deg[v], 1);  // the arc's position in coF(v)
    }
    if (e % K == K - 1)
        row_thresholds(e / K, key[e], v, tau, idxK, negH, nx, smax_bits, iv, bound_c, cmp, meta, Ex);
}

// The thresholds alone, from another graph of the same rows (the second phase
// of a split round): one thread per row.
__global__ void thresholds_kernel(const int32_t *__restrict__ idx, const double *__restrict__ key, int64_t n, int K,
                                  double *__restrict__ tau, int32_t *__restrict__ idxK, const double *__restrict__ negH,
                                  const double *__restrict__ nx, const unsigned long long *__restrict__ smax_bits,
                                  InstView iv, double bound_c, int cmp, RowMeta *__restrict__ meta,
                                  double *__restrict__ Ex)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int64_t e = x * K + (K - 1);
    row_thresholds(x, key[e], idx[e], tau, idxK, negH, nx, smax_bits, iv, bound_c, cmp, meta, Ex);
}

// Exclusive scan of the int32 degrees into int64 offsets, in three passes over
// tiles of kScanTile elements.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t s = (lane < kScanThreads / 32) ? wsum[lane] : 0;
        int64_t si = s;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < kScanThreads / 32) wsum[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    int64_t r = incl - v + wsum[w];
    __syncthreads();
    return r;
}

__global__ void scan_tiles_kernel(const int32_t *__restrict__ deg, const int32_t *__restrict__ deg_mut, int64_t n,
                                  int64_t *__restrict__ tile_sum)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t s = 0;
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += deg[base + i] + (deg_mut ? deg_mut[base + i] : 0);
    __shared__ int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void scan_sums_kernel(int64_t *__restrict__ tile_sum, int64_t ntiles, int64_t *__restrict__ off,
                                 int64_t n)
{
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = (i < ntiles) ? tile_sum[i] : 0;
        const int64_t ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void scan_apply_kernel(const int32_t *__restrict__ deg, const int32_t *__restrict__ deg_mut, int64_t n,
                                  const int64_t *__restrict__ tile_off,
                                  int64_t *__restrict__ off, RowMeta *__restrict__ meta, int K)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t s = 0;
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < n) ? deg[base + i] + (deg_mut ? deg_mut[base + i] : 0) : 0;
        s += v[i];
    }
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot) + tile_off[blockIdx.x];
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) {
            off[base + i] = run;
            if (meta) meta[base + i].boff = (long long)K * K * (base + i) + (long long)(K + 1) * run;
        }
        run += v[i];
    }
}

// One thread per arc x -> v: x goes to coF(v) at the position the count pass
// drew for the arc.  The order inside a list is not fixed; every consumer
// treats the list as a set.  With flag (incremental proposals), the arc's
// new-flag goes with it.
__global__ void csr_fill_kernel(const int32_t *__restrict__ idx, const int32_t *__restrict__ slot, int64_t n, int K,
                                const int64_t *__restrict__ off, int32_t *__restrict__ cof,
                                const uint8_t *__restrict__ flag, uint8_t *__restrict__ cof_new)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * K) return;
    const int32_t v = idx[e];
    if (v < 0 || v >= n) return;
    const int32_t sl = slot[e];
    const int64_t q = sl >= 0 ? off[v] + sl : off[v + 1] + sl;  // mutual arcs from the end
    cof[q] = (int32_t)(e / K);
    if (flag) cof_new[q] = flag[e];
}

cudaError_t launch_reverse_csr(knnd_handle *h, const int32_t *idx, const double *key)
{
    const int64_t n = h->n;
    const int K = h->K;
    const int64_t E = n * K;
    const int threads = 256;
    const unsigned eblocks = (unsigned)((E + threads - 1) / threads);
    cudaMemsetAsync(h->deg, 0, sizeof(int32_t) * n, h->stream);
    int32_t *deg_mut = (h->csr_mutual && join_runs_tma(h)) ? h->deg_mut : nullptr;  // mutual arcs apart
    if (deg_mut) cudaMemsetAsync(deg_mut, 0, sizeof(int32_t) * n, h->stream);
    const bool mixed = h->prec != KNND_PREC_FP64;
    csr_count_kernel<<<eblocks, threads, 0, h->stream>>>(idx, key, n, K, h->deg, h->slot, h->tau, h->idxK, h->negH,
                                                         h->nx,
                                                         h->smax_bits, h->iv, h->bound_c, h->prm.comparator,
                                                         mixed ? h->meta : nullptr,
                                                         h->Ex, h->err, deg_mut);
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    scan_tiles_kernel<<<(unsigned)ntiles, kScanThreads, 0, h->stream>>>(h->deg, deg_mut, n, h->scan_tmp);
    scan_sums_kernel<<<1, kScanThreads, 0, h->stream>>>(h->scan_tmp, ntiles, h->cof_off, n);
    scan_apply_kernel<<<(unsigned)ntiles, kScanThreads, 0, h->stream>>>(h->deg, deg_mut, n, h->scan_tmp,
                                                                        h->cof_off, mixed ? h->meta : nullptr, K);
    csr_fill_kernel<<<eblocks, threads, 0, h->stream>>>(idx, h->slot, n, K, h->cof_off, h->cof, h->round_flag,
                                                        h->cof_new);
    h->launches += 5;
    return cudaGetLastError();
}

cudaError_t launch_thresholds(knnd_handle *h, const int32_t *idx, const double *key)
{
    const int threads = 256;
    const bool mixed = h->prec != KNND_PREC_FP64;
    thresholds_kernel<<<(unsigned)((h->n + threads - 1) / threads), threads, 0, h->stream>>>(
        idx, key, h->n, h->K, h->tau, h->idxK, h->negH, h->nx, h->smax_bits, h->iv, h->bound_c, h->prm.comparator,
        mixed ? h->meta : nullptr, h->Ex);
    h->launches += 1;
    return cudaGetLastError();
}

}  // namespace knnd
