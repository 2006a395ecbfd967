// Measured arithmetic peaks for the roofline of the compute-bound kernels.
//
// The pair kernel (FP32 FMA pipe), its FP64 form and the FP64 preconditioner
// factorisations are bound by arithmetic, not memory, so their roofline
// denominator is the chip's FMA rate.  This file measures it on the device
// the context runs on, at the clocks of the moment: every thread runs
// kChains independent FMA recurrences x <- x m + b (no memory traffic in the
// loop, enough independent work to cover the pipe's latency), the launch
// fills every SM with 2,048 threads, and the rate is the counted FMAs over
// the launch's CUDA-event duration (best of three launches after a warm-up).
#include <algorithm>

#include "mb_internal.cuh"

namespace mb {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

// FP32: paired fma.rn.f32x2, two FMAs per instruction, so the FMA pipe (not
// instruction issue) is the limit.
__global__ void __launch_bounds__(kThreads) fma_rate_f32_kernel(float *out, float seed, int iters)
{
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = make_float2(seed + (float)c, seed - (float)(threadIdx.x & 7));
    const float2 m = make_float2(0.9375f, 0.9375f), b = make_float2(0.0625f, 0.0625f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
    if (s == -1.0f) out[threadIdx.x] = s;  // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) fma_rate_f64_kernel(double *out, double seed, int iters)
{
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + (double)c - (double)(threadIdx.x & 7);
    const double m = 0.9375, b = 0.0625;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == -1.0) out[threadIdx.x] = s;
}

}  // namespace
}  // namespace mb

using namespace mb;

extern "C" mb_status mb_measure_fma_rate(mb_context *ctx, mb_precision prec, double *flops_per_s,
                                         void *stream)
{
    if (!ctx) return MB_EINVAL;
    ctx->err.clear();
    if (!flops_per_s) return set_err(ctx, MB_EINVAL, "null output pointer");
    if (prec != MB_FP32_KAHAN && prec != MB_FP64)
        return set_err(ctx, MB_EINVAL, "FMA rate is measured for MB_FP32_KAHAN or MB_FP64");
    MB_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const bool f32 = prec == MB_FP32_KAHAN;
    const int grid = ctx->sm_count * (2048 / kThreads);
    // about 30 ms per launch at the nominal rates (80 TFLOP/s FP32, 1 TFLOP/s FP64)
    const int iters = f32 ? 16384 : 512;
    const double fma_per_thread = (double)iters * kUnroll * kChains * (f32 ? 2.0 : 1.0);
    const double flops = 2.0 * fma_per_thread * kThreads * (double)grid;
    MB_TRY(ensure(ctx, ctx->sol_small, sizeof(double) * kThreads, "FMA-rate probe"));
    cudaEvent_t e0, e1;
    MB_CUDA_TRY(ctx, cudaEventCreate(&e0));
    MB_CUDA_TRY(ctx, cudaEventCreate(&e1));
    float best = 0.f;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < 4 && err == cudaSuccess; ++k) {
        cudaEventRecord(e0, s);
        if (f32)
            fma_rate_f32_kernel<<<grid, kThreads, 0, s>>>((float *)ctx->sol_small.ptr, 1.0f, iters);
        else
            fma_rate_f64_kernel<<<grid, kThreads, 0, s>>>((double *)ctx->sol_small.ptr, 1.0, iters);
        count_launch();
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (k > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_err(ctx, err, "FMA-rate probe");
    MB_CUDA_TRY(ctx, cudaGetLastError());
    *flops_per_s = flops / (1e-3 * (double)best);
    return MB_OK;
}
