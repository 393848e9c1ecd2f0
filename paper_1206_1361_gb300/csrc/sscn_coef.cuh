// sscn_coef.cuh -- coefficient tables as the kernels see them.
//
// FP64 path: a complex coefficient is a double2.  Complex64 path: a float4
// (hi.x, hi.y, lo.x, lo.y) with hi the FP32 rounding of the FP64 value and lo
// the FP32 rounding of the remainder, so hi + lo carries the coefficient to
// ~2^-48.  A product v * (hi + lo) is rounded once, like v * hi, but the
// coefficient itself is no longer off by an FP32 rounding: a table reused
// every step would otherwise perturb the Crank-Nicolson operator (and the
// unit-modulus potential factors) by the same ~2^-24 at every step, and in
// real time that breaks the norm conservation linearly in the step count.
#pragma once

template <typename T> struct Coef;
template <> struct Coef<double> { using t = double2; };
template <> struct Coef<float> { using t = float4; };

// complex v * coefficient f
__device__ __forceinline__ double2 cmulc(double2 v, double2 f)
{
    return make_double2(fma(v.x, f.x, -v.y * f.y), fma(v.x, f.y, v.y * f.x));
}
__device__ __forceinline__ float2 cmulc(float2 v, float4 f)
{
    const float lx = fmaf(v.x, f.z, -v.y * f.w), ly = fmaf(v.x, f.w, v.y * f.z);
    return make_float2(fmaf(v.x, f.x, fmaf(-v.y, f.y, lx)), fmaf(v.x, f.y, fmaf(v.y, f.x, ly)));
}

// v * the hi part alone: for recurrences whose coefficient rounding is
// scaled down by a small right-hand side (the increment form), where one
// FP32 rounding of the coefficient is far below the result's own rounding
__device__ __forceinline__ float2 cmulc_hi(float2 v, float4 f)
{
    return make_float2(fmaf(v.x, f.x, -v.y * f.y), fmaf(v.x, f.y, v.y * f.x));
}
__device__ __forceinline__ float rmulc_hi(float v, float4 f) { return v * f.x; }

// real part of a coefficient (imaginary time: tables are real) times v
__device__ __forceinline__ double rmulc(double v, double2 f) { return v * f.x; }
__device__ __forceinline__ float rmulc(float v, float4 f) { return fmaf(v, f.x, v * f.z); }

// real part as one number of the working precision
__device__ __forceinline__ double coef_re(double2 f) { return f.x; }
__device__ __forceinline__ float coef_re(float4 f) { return f.x + f.z; }
