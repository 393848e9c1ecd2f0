// sscn_accum.cuh -- per-thread partial sums for the FP64 reductions.
//
// Acc<double> adds in FP64.  Acc<float> serves the complex64 form, whose
// per-point terms are FP32 products of FP32 values: a thread's run of terms
// (a grid line, or a lane's points of several lines) is summed with Kahan's
// compensated summation in FP32 -- error within about two FP32 ulps of the
// partial, independent of the number of terms, below the rounding of the
// complex64 state itself -- and handed to the FP64 reductions across threads
// and blocks.  On GB300 an FP64 add costs as much FP64-pipe
// time as ~60 FP32 operations, so this keeps the complex64 kernels off the
// FP64 pipe.
#pragma once

template <typename T> struct Acc;

template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add_sq2(double a, double b) { s = fma(a, a, fma(b, b, s)); }
    __device__ __forceinline__ double get() const { return s; }
};

template <> struct Acc<float> {
    float s = 0.f, c = 0.f;                  // c: running compensation
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b) { add(a * b); }
    __device__ __forceinline__ void add_sq2(float a, float b) { add(fmaf(a, a, b * b)); }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Warp sum of the values s - c (Kahan pairs from Acc<float>) in FP32, the
// rounding of every addition carried along (TwoSum): the total in FP64,
// valid in lane 0.  FP64 adds across a warp would cost 16 FP64-pipe clocks
// each on GB300.
__device__ __forceinline__ double warp_sum_comp(float s, float c)
{
    float hi = s, lo = -c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const float t = hi + h2, z = t - hi;
        const float e = (hi - (t - z)) + (h2 - z);
        hi = t;
        lo = lo + l2 + e;
    }
    return (double)hi + (double)lo;
}
