// peak.cu -- knnd_fma_peak: the issue-limited rate of the FMA pipes the join
// forms run on, measured on the device in use.  Measurement support for the
// roofline fractions of the FP32 filter (FFMA, packed FFMA2) and of the FP64
// form (DFMA); not part of the method.
//
// Every thread runs kChains independent fma chains for `iters` steps on
// operands the compiler cannot fold (read from the sink, which holds zeros),
// and writes one sum back so that nothing is dead code.  The grid is
// blocks_per_sm blocks of 256 threads on every SM.  FLOPs counted: 2 per fma
// (4 per packed FFMA2).
#include "knnd_internal.cuh"

namespace knnd {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_f32_kernel(int64_t iters, float *sink)
{
    const float a = 1.0f + sink[0], b = 1e-7f * (1.0f + sink[1]);
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (float)(threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __fmaf_rn(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == -1.0f) sink[2] = s;  // never true for these operands; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) fma_f32x2_kernel(int64_t iters, float *sink)
{
    const float2 a = make_float2(1.0f + sink[0], 1.0f + sink[0]);
    const float2 b = make_float2(1e-7f * (1.0f + sink[1]), 2e-7f * (1.0f + sink[1]));
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = make_float2((float)(threadIdx.x + c), (float)c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
    if (s == -1.0f) sink[2] = s;
}

__global__ void __launch_bounds__(kPeakThreads) fma_f64_kernel(int64_t iters, float *sink)
{
    const double a = 1.0 + sink[0], b = 1e-15 * (1.0 + sink[1]);
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (double)(threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __fma_rn(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == -1.0) sink[2] = (float)s;
}

}  // namespace
}  // namespace knnd

extern "C" knnd_status knnd_fma_peak(int32_t kind, int32_t blocks_per_sm, int64_t iters, float *sink,
                                     double *flops, float *ms, void *stream)
{
    if (kind < 0 || kind > 2 || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !sink || !flops || !ms)
        return KNND_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return KNND_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KNND_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KNND_ECUDA;
    }
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    cudaEventRecord(e0, st);
    if (kind == 0) knnd::fma_f32_kernel<<<grid, knnd::kPeakThreads, 0, st>>>(iters, sink);
    else if (kind == 1) knnd::fma_f32x2_kernel<<<grid, knnd::kPeakThreads, 0, st>>>(iters, sink);
    else knnd::fma_f64_kernel<<<grid, knnd::kPeakThreads, 0, st>>>(iters, sink);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return KNND_ECUDA;
    *ms = t;
    *flops = 2.0 * (kind == 1 ? 2.0 : 1.0) * (double)grid * knnd::kPeakThreads * knnd::kChains * (double)iters;
    return KNND_OK;
}
