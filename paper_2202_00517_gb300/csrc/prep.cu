// prep.cu -- per-build precompute (log table, -H(x), FP32 copies, error-bound
// scale), the initial random K-out graph (Sec. 3.2) and the friend clustering
// sample (Sec. 3.3).
#include <cfloat>

#include "knnd_internal.cuh"

namespace knnd {

// ---------------------------------------------------------------------------
// Precompute (Sec. 2.2 rewritten as key(x, y) = negH(x) - <x, log y>):
// one thread per point.  L = log(x) in FP64 (CUDA's double-precision log),
// negH = sum_i x_i L_i as a sequential fma chain from 0, nx = sum_i |x_i|,
// and the largest |L| over all coordinates (the FP32 error-bound scale).
// Coordinates that are not finite or not > 0 set kErrDomain.
// ---------------------------------------------------------------------------
// Points: pts + x * ld, or (several instances) the row x - base[i] of
// instance i = iv.of[x] at ptrs[i] with row stride lds[i].
// mode 0: the KL comparators (L = log x, negH = sum x log x).  Comparators on the
// coordinates themselves (mode 1: squared Euclidean; mode 2: inner product): L is
// a copy of the coordinates and negH holds |x|^2 (fma chain from 0) for the
// first, 0 for the second; coordinates need only be finite.
template <typename T>
__global__ void precompute_kernel(const T *__restrict__ pts, int64_t ld, const void *const *ptrs,
                                  const int64_t *lds, InstView iv, int mode, int64_t n, int m, int MP,
                                  double *__restrict__ X64, double *__restrict__ L64, float *__restrict__ X32,
                                  float *__restrict__ L32, double *__restrict__ negH, double *__restrict__ nx,
                                  unsigned long long *smax_bits, int32_t *err)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double lmax = 0.0, hmax = 0.0, nmax = 0.0;
    if (x < n) {
        double acc = 0.0, s = 0.0;
        bool bad = false;
        const T *row;
        if (iv.of) {
            const int i = iv.of[x];
            row = static_cast<const T *>(ptrs[i]) + (x - iv.base[i]) * lds[i];
        } else {
            row = pts + x * ld;
        }
        for (int i = 0; i < MP; ++i) {
            double v = 0.0, l = 0.0;
            if (i < m) {
                v = (double)row[i];
                if (mode ? !(fabs(v) <= DBL_MAX) : (!(v > 0.0) || !(v <= DBL_MAX))) {
                    bad = true;
                    v = 1.0;  // keep the tables finite; the call reports EDOMAIN
                }
                l = mode ? v : log(v);
                if (mode != 2) acc = __fma_rn(v, l, acc);
                s += fabs(v);
                lmax = fmax(lmax, fabs(l));
            }
            X64[x * MP + i] = v;
            L64[x * MP + i] = l;
            X32[x * MP + i] = __double2float_rn(v);
            L32[x * MP + i] = __double2float_rn(l);
        }
        negH[x] = acc;
        nx[x] = s;
        hmax = fabs(acc);
        nmax = s;
        if (bad) atomicOr(err, kErrDomain);
    }
    if (iv.of) {  // several instances: one set of maxima each
        if (x < n) {
            unsigned long long *mx = smax_bits + 3 * (int64_t)iv.of[x];
            atomicMax(&mx[0], (unsigned long long)__double_as_longlong(lmax));
            atomicMax(&mx[1], (unsigned long long)__double_as_longlong(hmax));
            atomicMax(&mx[2], (unsigned long long)__double_as_longlong(nmax));
        }
        return;
    }
    // block maxima -> one atomicMax each on the (monotone) bits of non-negative doubles
    for (int o = 16; o > 0; o >>= 1) {
        lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        hmax = fmax(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
        nmax = fmax(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    }
    __shared__ double wmax[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        wmax[0][w] = lmax;
        wmax[1][w] = hmax;
        wmax[2][w] = nmax;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, wmax[threadIdx.x][i]);
        atomicMax(&smax_bits[threadIdx.x], (unsigned long long)__double_as_longlong(b));
    }
}

// 0: log tables (the KL comparators); 1: squared Euclidean; 2: inner product
static int coord_mode(int cmp)
{
    return cmp == KNND_CMP_SQEUCLIDEAN ? 1 : (cmp == KNND_CMP_INNER ? 2 : 0);
}

cudaError_t launch_precompute(knnd_handle *h, const void *points, int64_t ld)
{
    return launch_precompute_from(h, points, ld, nullptr, nullptr);
}

cudaError_t launch_precompute_from(knnd_handle *h, const void *points, int64_t ld, const void *const *ptrs,
                                   const int64_t *lds)
{
    const int threads = 256;
    const int64_t blocks = (h->n + threads - 1) / threads;
    cudaMemsetAsync(h->smax_bits, 0, sizeof(unsigned long long) * 3 * (h->ninst > 0 ? h->ninst : 1), h->stream);
    if (h->dtype == KNND_F32)
        precompute_kernel<float><<<(unsigned)blocks, threads, 0, h->stream>>>(
            (const float *)points, ld, ptrs, lds, h->iv, coord_mode(h->prm.comparator), h->n, h->m, h->MP,
            h->X64, h->L64, h->X32, h->L32,
            h->negH, h->nx, h->smax_bits, h->err);
    else
        precompute_kernel<double><<<(unsigned)blocks, threads, 0, h->stream>>>(
            (const double *)points, ld, ptrs, lds, h->iv, coord_mode(h->prm.comparator), h->n, h->m, h->MP,
            h->X64, h->L64, h->X32, h->L32,
            h->negH, h->nx, h->smax_bits, h->err);
    h->launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fma chain over i of X64[x]_i * L64[y]_i, from 0 (padding terms are exact no-ops).
__device__ __forceinline__ double dot_fp64(const double *__restrict__ X64, const double *__restrict__ L64, int MP,
                                           int64_t x, int64_t y)
{
    const double2 *xr = reinterpret_cast<const double2 *>(X64 + x * MP);
    const double2 *lr = reinterpret_cast<const double2 *>(L64 + y * MP);
    double acc = 0.0;
    for (int i = 0; i < MP / 2; ++i) {
        double2 a = xr[i], b = lr[i];
        acc = __fma_rn(a.x, b.x, acc);
        acc = __fma_rn(a.y, b.y, acc);
    }
    return acc;
}

// The comparator's canonical FP64 key: KL negH(x) - <x, log y>; reverse KL the
// same with the roles swapped; squared Euclidean (|x|^2 - 2 <x, y>) + |y|^2 (L64
// then holds the coordinates and negH the squared norms); inner product the KL
// form with L64 the coordinates and negH = 0, i.e. 0 - <x, y>.
__device__ __forceinline__ double key_cmp(int cmp, const double *__restrict__ X64, const double *__restrict__ L64,
                                          const double *__restrict__ negH, int MP, int64_t x, int64_t y)
{
    if (cmp == KNND_CMP_KL_REVERSE) return negH[y] - dot_fp64(X64, L64, MP, y, x);
    if (cmp == KNND_CMP_SQEUCLIDEAN) return (negH[x] - 2.0 * dot_fp64(X64, L64, MP, x, y)) + negH[y];
    return negH[x] - dot_fp64(X64, L64, MP, x, y);
}

// ---------------------------------------------------------------------------
// Initial random K-out graph (Sec. 3.2): one thread per point x.  Friends are
// drawn from Philox stream (seed, x, 0, kTagInit): y' uniform in [0, n-1),
// y = y' + (y' >= x), a repeat drawn again.  Rows sorted by (key, idx).
// ---------------------------------------------------------------------------
// cmp: the comparator (KNND_CMP_*), see key_cmp.
__global__ void init_graph_kernel(int64_t n, int K, int MP, const double *__restrict__ X64,
                                  const double *__restrict__ L64, const double *__restrict__ negH, uint64_t seed,
                                  InstView iv, int cmp, int32_t *__restrict__ idx, double *__restrict__ key,
                                  uint8_t *__restrict__ flag)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    // several instances: draws use the instance's seed, local indices and size
    int64_t base = 0, nl = n;
    if (iv.of) {
        const int i = iv.of[x];
        base = iv.base[i];
        nl = iv.n[i];
        seed = iv.seed[i];
    }
    const int64_t xl = x - base;
    int ids[KNND_MAX_K];
    double ks[KNND_MAX_K];
    Philox ph(seed, (uint32_t)xl, 0u, kTagInit);
    int cnt = 0;
    while (cnt < K) {
        uint32_t yp = ph.bounded((uint32_t)(nl - 1));
        int y = (int)(base + (int64_t)yp + ((int64_t)yp >= xl ? 1 : 0));
        bool dup = false;
        for (int t = 0; t < cnt; ++t) dup |= (ids[t] == y);
        if (dup) continue;
        ids[cnt++] = y;
    }
    for (int t = 0; t < K; ++t)
        ks[t] = key_cmp(cmp, X64, L64, negH, MP, x, ids[t]);
    for (int t = 1; t < K; ++t) {  // insertion sort by (key, idx)
        double kk = ks[t];
        int ii = ids[t];
        int s = t - 1;
        while (s >= 0 && lex_less(kk, ii, ks[s], ids[s])) {
            ks[s + 1] = ks[s];
            ids[s + 1] = ids[s];
            --s;
        }
        ks[s + 1] = kk;
        ids[s + 1] = ii;
    }
    for (int t = 0; t < K; ++t) {
        idx[x * K + t] = ids[t];
        key[x * K + t] = ks[t];
        if (flag) flag[x * K + t] = 1;
    }
}

cudaError_t launch_init_graph(knnd_handle *h, uint64_t seed, int32_t *idx, double *key, uint8_t *newflag)
{
    const int threads = 128;
    const int64_t blocks = (h->n + threads - 1) / threads;
    init_graph_kernel<<<(unsigned)blocks, threads, 0, h->stream>>>(h->n, h->K, h->MP, h->X64, h->L64, h->negH,
                                                                   seed, h->iv, h->prm.comparator, idx, key, newflag);
    h->launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Friend clustering sample (Sec. 3.3): thread per sample s, stream
// (seed, s, round, kTagFcc): x uniform in [0, n), i uniform in [0, K),
// j' uniform in [0, K-1), j = j' + (j' >= i).  Hit when z = F(x)[j] is a friend
// of y = F(x)[i] or y is a friend of z.  Indices outside [0, n) set kErrIndex
// and count as misses.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool row_has(const int32_t *__restrict__ idx, int K, int64_t a, int32_t b)
{
    bool f = false;
    for (int t = 0; t < K; ++t) f |= (idx[a * K + t] == b);
    return f;
}

__global__ void fcc_kernel(const int32_t *__restrict__ idx, int64_t n, int K, uint64_t seed, int32_t round,
                           int32_t S, int64_t *hits, int32_t *err, const LoopState *loop)
{
    if (loop) {  // a round of the device-driven loop
        seed = loop->seed;
        round = loop->round;
    }
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int hit = 0;
    if (s < S) {
        Philox ph(seed, (uint32_t)s, (uint32_t)round, kTagFcc);
        int64_t x = ph.bounded((uint32_t)n);
        int i = (int)ph.bounded((uint32_t)K);
        int jp = (int)ph.bounded((uint32_t)(K - 1));
        int j = jp + (jp >= i ? 1 : 0);
        int32_t y = idx[x * K + i], z = idx[x * K + j];
        if (y < 0 || y >= n || z < 0 || z >= n) {
            atomicOr(err, kErrIndex);
        } else {
            hit = (row_has(idx, K, y, z) || row_has(idx, K, z, y)) ? 1 : 0;
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, hit);
    __shared__ int wsum[32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        if (t) atomicAdd((unsigned long long *)hits, (unsigned long long)t);
    }
}

// Several instances: thread (i, s) draws sample s of instance i from its own
// stream (seed_i, s, round, kTagFcc) over its local indices; hits go to the
// instance's counter.  Stopped instances draw nothing.
__global__ void fcc_batch_kernel(const int32_t *__restrict__ idx, int K, InstView iv, int32_t ninst, int32_t round,
                                 int32_t S, int32_t *err, const int32_t *round_dev)
{
    if (round_dev) round = *round_dev;  // a round of a device-driven loop
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ninst * S) return;
    const int i = (int)(t / S);
    const int s = (int)(t - (int64_t)i * S);
    if (!iv.active[i]) return;
    const int64_t base = iv.base[i];
    const int64_t nl = iv.n[i];
    Philox ph(iv.seed[i], (uint32_t)s, (uint32_t)round, kTagFcc);
    const int64_t x = base + ph.bounded((uint32_t)nl);
    const int a = (int)ph.bounded((uint32_t)K);
    const int bp = (int)ph.bounded((uint32_t)(K - 1));
    const int b = bp + (bp >= a ? 1 : 0);
    const int32_t y = idx[x * K + a], z = idx[x * K + b];
    if (y < base || y >= base + nl || z < base || z >= base + nl) {
        atomicOr(err, kErrIndex);
        return;
    }
    if (row_has(idx, K, y, z) || row_has(idx, K, z, y))
        atomicAdd((unsigned long long *)&iv.cnt[(int64_t)i * kCntNum + kCntHits], 1ull);
}

cudaError_t launch_fcc_batch(knnd_handle *h, const int32_t *idx, int32_t round, const int32_t *round_dev)
{
    const int threads = 256;
    const int64_t total = (int64_t)h->ninst * h->prm.fcc_samples;
    fcc_batch_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, h->stream>>>(
        idx, h->K, h->iv, h->ninst, round, h->prm.fcc_samples, h->err, round_dev);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_fcc(knnd_handle *h, const int32_t *idx, uint64_t seed, int32_t round, int64_t *hits_out,
                       const LoopState *loop)
{
    const int threads = 256;
    const int S = h->prm.fcc_samples;
    cudaMemsetAsync(hits_out, 0, sizeof(int64_t), h->stream);
    fcc_kernel<<<(S + threads - 1) / threads, threads, 0, h->stream>>>(idx, h->n, h->K, seed, round, S, hits_out,
                                                                       h->err, loop);
    h->launches += 1;
    return cudaGetLastError();
}

// Raw Philox4x32-10 blocks: thread i maps counter ctr_key[6i..6i+3] under key
// ctr_key[6i+4..6i+5] to out[4i..4i+3] with the routine every draw uses.
__global__ void philox_kernel(const uint32_t *__restrict__ ck, uint32_t *__restrict__ out, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t *c = ck + 6 * i;
    Philox ph(((uint64_t)c[5] << 32) | c[4], c[0], c[1], c[2]);
    ph.block = c[3];
    for (int w = 0; w < 4; ++w) out[4 * i + w] = ph.next();
}

}  // namespace knnd

extern "C" knnd_status knnd_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int64_t count, void *stream)
{
    if (count < 0 || count >= ((int64_t)1 << 31)) return KNND_EINVAL;
    if (count == 0) return KNND_OK;
    if (!ctr_key || !out) return KNND_EINVAL;
    const int threads = 128;
    knnd::philox_kernel<<<(unsigned)((count + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
        ctr_key, out, count);
    return cudaGetLastError() == cudaSuccess ? KNND_OK : KNND_ECUDA;
}
