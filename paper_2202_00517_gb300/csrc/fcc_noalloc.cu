// fcc_noalloc.cu -- knnd_fcc_noalloc: the friend clustering sample of
// knnd_fcc, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where the device memory is owned by someone
// else -- an application whose memory pool or caching allocator already
// reserves nearly all of the GPU (a raw cudaMalloc would fail or fragment
// it), a serving loop that forbids allocation after start-up to keep its
// latency predictable, or a plug-in whose host requires every allocation to
// go through the host's own allocator.  Such a caller cannot create a
// knnd_handle (knnd_create allocates the workspace), but it can still run its
// own descent loop and needs the statistical stop test on its graph.
//
// The scratch this sample needs (one partial hit count per block of samples
// and an error word) lives in the file-scope device array below instead of in
// a handle.  Its size is fixed: KNND_NOALLOC_MAX_SAMPLES samples at most.
// Every GPU that loads the library holds the array until the process exits.
// All calls on one device share it and it keeps the last call's contents, so
// calls whose work overlaps on the GPU (different streams, or different host
// threads, without ordering between them) race and may return wrong counts.
#include "knnd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = (KNND_NOALLOC_MAX_SAMPLES + kThreads - 1) / kThreads;
// [0, 8): error word (int32) + pad; [256, 256 + 8 * kMaxBlocks): partial hit counts
constexpr size_t kPartialsOffset = 256;
constexpr size_t kScratchBytes = kPartialsOffset + sizeof(long long) * kMaxBlocks;

static __device__ __align__(256) unsigned char g_fcc_scratch[kScratchBytes];

// Device address of g_fcc_scratch in the current device's current context.
// In host code the symbol itself is only a host-side stand-in.  The address is
// looked up on every call (a host-side query, not a stream operation), never
// cached: a context torn down and made again (cudaDeviceReset) reloads the
// module, and an address kept from the old context would point nowhere.
knnd_status scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fcc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        (void)cudaGetLastError();
        return KNND_ECUDA;
    }
    *out = p;
    return KNND_OK;
}

__device__ __forceinline__ bool row_contains(const int32_t *__restrict__ idx, int K, int64_t a, int32_t b)
{
    bool f = false;
    for (int t = 0; t < K; ++t) f |= (idx[a * K + t] == b);
    return f;
}

// Same draws and hit rule as the handle's sample; each block writes its hit
// count to partials[blockIdx.x] instead of adding to the output.
__global__ void fcc_partial_kernel(const int32_t *__restrict__ idx, int64_t n, int K, uint64_t seed, int32_t round,
                                   int32_t S, long long *__restrict__ partials, int32_t *err)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int hit = 0;
    if (s < S) {
        knnd::Philox ph(seed, (uint32_t)s, (uint32_t)round, knnd::kTagFcc);
        const int64_t x = ph.bounded((uint32_t)n);
        const int i = (int)ph.bounded((uint32_t)K);
        const int jp = (int)ph.bounded((uint32_t)(K - 1));
        const int j = jp + (jp >= i ? 1 : 0);
        const int32_t y = idx[x * K + i], z = idx[x * K + j];
        if (y < 0 || y >= n || z < 0 || z >= n)
            atomicOr(err, 1);
        else
            hit = (row_contains(idx, K, y, z) || row_contains(idx, K, z, y)) ? 1 : 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    __shared__ int wsum[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += wsum[w];
        partials[blockIdx.x] = t;
    }
}

// Sums the partial counts (fixed order, one block) into *hits; -1 when some
// sampled friend index was outside [0, n).
__global__ void fcc_sum_kernel(const long long *__restrict__ partials, int nblocks, const int32_t *err,
                               int64_t *hits)
{
    long long t = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += partials[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __shared__ long long wsum[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long total = 0;
        for (int w = 0; w < kThreads / 32; ++w) total += wsum[w];
        *hits = (*err != 0) ? -1 : (int64_t)total;
    }
}

}  // namespace

extern "C" knnd_status knnd_fcc_noalloc(const int32_t *idx, int64_t n, int32_t K, uint64_t seed, int32_t round,
                                        int32_t samples, int64_t *hits, void *stream)
{
    if (!idx || !hits || round < 0 || samples < 1) return KNND_EINVAL;
    if (n < 3 || n >= ((int64_t)1 << 31) || K < 2 || K > KNND_MAX_K || (int64_t)K >= n) return KNND_EINVAL;
    if (samples > KNND_NOALLOC_MAX_SAMPLES) return KNND_EOVERFLOW;
    void *base = nullptr;
    knnd_status s = scratch_address(&base);
    if (s) return s;
    int32_t *err = reinterpret_cast<int32_t *>(base);
    long long *partials = reinterpret_cast<long long *>(static_cast<unsigned char *>(base) + kPartialsOffset);
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (samples + kThreads - 1) / kThreads;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);  // the array keeps the last call's value
    if (e == cudaSuccess) {
        fcc_partial_kernel<<<blocks, kThreads, 0, st>>>(idx, n, K, seed, round, samples, partials, err);
        fcc_sum_kernel<<<1, kThreads, 0, st>>>(partials, blocks, err, hits);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) return KNND_OK;
    return KNND_ECUDA;
}
