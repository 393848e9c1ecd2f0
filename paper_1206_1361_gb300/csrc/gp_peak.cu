// gp_peak.cu -- arithmetic-rate microbenchmarks: the denominators of the
// "alu" rooflines of the sweep kernels (FP64 fused multiply-add for the
// complex128 form, FP32 and packed FP32x2 fused multiply-add for the
// complex64 and float-float forms).
//
// Each thread runs kChains independent multiply-add chains, x <- x * b + c,
// with b slightly below 1 so nothing overflows; the chains are independent so
// the pipe, not the latency of one chain, sets the rate.  One launch covers
// kBlocksPerSm CTAs per SM of 256 threads; the result is the best of kRuns
// timed launches (CUDA events) after one warm-up launch.

#include <cstdint>
#include <cuda_runtime.h>

#include "gp.h"
#include "sscn_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kRuns = 3;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_peak(double *out, long long iters, double b, double c)
{
    if constexpr (KIND == GP_PEAK_FP64_FMA) {
        double x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3 + j;
        for (long long i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, c);
        }
        double s = 0;
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j];
        if (s == 12345.678) out[0] = s;   // keeps the chains live
    } else if constexpr (KIND == GP_PEAK_FP32_FMA) {
        const float bf = (float)b, cf = (float)c;
        float x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3f + j;
        for (long long i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], bf, cf);
        }
        float s = 0;
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j];
        if (s == 12345.678f) out[0] = s;
    } else {
        const float2 bf = make_float2((float)b, (float)b), cf = make_float2((float)c, (float)c);
        float2 x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = make_float2(threadIdx.x * 1e-3f + j, j + 0.5f);
        for (long long i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], bf, cf);
        }
        float s = 0;
#pragma unroll
        for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
        if (s == 12345.678f) out[0] = s;
    }
}

template <int KIND>
cudaError_t run_peak(long long iters, int sms, double *buf, cudaStream_t st, float *ms_best)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const dim3 grid(sms * kBlocksPerSm);
    *ms_best = 0.f;
    for (int r = 0; r <= kRuns && e == cudaSuccess; ++r) {
        k_peak<KIND><<<grid, kThreads, 0, st>>>(buf, r == 0 ? iters / 8 + 1 : iters, 0.999999, 1e-7);
        e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) break;
        k_peak<KIND><<<grid, kThreads, 0, st>>>(buf, iters, 0.999999, 1e-7);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = cudaEventRecord(e1, st);
        if (e != cudaSuccess) break;
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0;
        e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && (*ms_best == 0.f || ms < *ms_best)) *ms_best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" int gp_measure_peak(int kind, int64_t iters, double *tflops, double *ms)
{
    if (kind < GP_PEAK_FP64_FMA || kind > GP_PEAK_FP32X2_FMA || iters < 1 || !tflops) {
        gp::set_thread_error("gp_measure_peak: bad kind, iteration count or output pointer");
        return GP_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        gp::set_thread_error(cudaGetErrorString(e));
        return GP_ECUDA;
    }
    double *buf = nullptr;
    e = cudaMalloc(&buf, sizeof(double));
    if (e != cudaSuccess) {
        gp::set_thread_error("gp_measure_peak: cudaMalloc failed");
        return GP_ENOMEM;
    }
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    float best = 0.f;
    if (e == cudaSuccess) {
        if (kind == GP_PEAK_FP64_FMA) e = run_peak<GP_PEAK_FP64_FMA>(iters, sms, buf, st, &best);
        else if (kind == GP_PEAK_FP32_FMA) e = run_peak<GP_PEAK_FP32_FMA>(iters, sms, buf, st, &best);
        else e = run_peak<GP_PEAK_FP32X2_FMA>(iters, sms, buf, st, &best);
        cudaStreamDestroy(st);
    }
    cudaFree(buf);
    if (e != cudaSuccess || best <= 0.f) {
        gp::set_thread_error(e != cudaSuccess ? cudaGetErrorString(e) : "gp_measure_peak: no timing");
        return GP_ECUDA;
    }
    // two flops per multiply-add, two multiply-adds per packed instruction
    const double fmas = (double)sms * kBlocksPerSm * kThreads * kChains * (double)iters *
                        (kind == GP_PEAK_FP32X2_FMA ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return GP_OK;
}
