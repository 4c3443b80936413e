// Arithmetic-pipe microbenchmarks of the GPU the echo path runs on: the
// denominators of the echo kernels' roofline (FP32 FMA, packed FP32x2 FMA, FP64
// FMA, and the special-function unit through __sinf), measured rather than taken
// from unit counts. Each kernel runs independent dependency chains per thread
// (enough of them to cover the pipe latency) on a grid of several CTAs per SM and
// writes one value per thread so that no chain is dead code.
#include <cuda_runtime.h>

#include "harm_peaks.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_kernel(int iters, float seed, float *out)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999999f, k = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma2_kernel(int iters, float seed, float *out)
{
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    const float2 m = make_float2(0.999999f, 0.999998f), k = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_kernel(int iters, float seed, float *out)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (double)seed + (double)(threadIdx.x + c);
    const double m = 0.999999999, k = 1e-12;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(256) sinf_kernel(int iters, float seed, float *out)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 0.01f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __sinf(a[c]);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int harm_peak_launch(int kind, int blocks, int iters, void *out_dev, void *stream)
{
    if (blocks < 1 || iters < 1 || !out_dev) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    float *out = (float *)out_dev;
    switch (kind) {
    case HARM_PEAK_FFMA: ffma_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, out); break;
    case HARM_PEAK_FFMA2: ffma2_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, out); break;
    case HARM_PEAK_DFMA: dfma_kernel<<<blocks, 256, 0, st>>>(iters, 1.0f, out); break;
    case HARM_PEAK_SINF: sinf_kernel<<<blocks, 256, 0, st>>>(iters, 0.5f, out); break;
    default: return 1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" long long harm_peak_ops(int kind, int blocks, int iters)
{
    const long long lanes = (long long)blocks * 256 * kChains * iters;
    switch (kind) {
    case HARM_PEAK_FFMA: return 2 * lanes;   // flops
    case HARM_PEAK_FFMA2: return 4 * lanes;  // flops (two FMAs per instruction)
    case HARM_PEAK_DFMA: return 2 * lanes;   // flops
    case HARM_PEAK_SINF: return lanes;       // __sinf evaluations
    default: return 0;
    }
}
