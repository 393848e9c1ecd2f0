// sscn_accum.cuh -- per-thread partial sums for the FP64 reductions.
//
// Acc<double> adds in FP64.  Acc<float> serves the complex64 form, whose
// per-point terms are FP32 products of FP32 values: a thread's run of terms
// (at most one grid line) is summed with Kahan's compensated summation in
// FP32 -- error within about two FP32 ulps of the partial, below the rounding
// of the complex64 state itself -- and handed to the FP64 reductions across
// threads, lines and blocks.  On GB300 an FP64 add costs as much FP64-pipe
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
