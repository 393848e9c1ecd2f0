// sscn_ff.cuh -- float-float ("double-single") arithmetic for the FP64-class
// form of the sweeps, on the FP32 pipe.
//
// A real number is carried as an unevaluated sum hi + lo of two FP32 values
// (about 48 significant bits).  The building blocks are the error-free
// transformations: Knuth's TwoSum (s + e == a + b exactly, s = fl(a + b),
// six additions, no condition on the operands), Dekker's Fast2Sum (three
// additions, for |a| >= |b|) and the FMA form of Dekker's TwoProduct
// (p + e == a b exactly, p = fl(a b), e = fma(a, b, -p)).
//
// A complex value (C) keeps its real and imaginary parts in the two lanes of
// packed FP32x2 registers -- hi = (re_hi, im_hi), lo = (re_lo, im_lo) -- so
// the same sequence of packed instructions (FADD2 / FMUL2 / FFMA2 on
// sm_100+) works on both parts.  On GB300 a packed instruction occupies the
// FP32 pipe for two cycles, so packing does not raise the FP32 rate; it
// halves the issue slots the arithmetic takes, leaving the other half for
// the shared-memory traffic, register moves and control of the sweep.
//
// Intermediate results are left unnormalised (lo may exceed half an ulp of
// hi by a few ulps, and after cancellation lo may be as large as hi): every
// later operation still forms each partial product of hi and lo, so the
// absolute error stays at ~2^-48 of the operands' magnitude.  Results that
// are stored (psi) are normalised with Fast2Sum.
#pragma once

#include <cuda_runtime.h>

#include "sscn_internal.h"

namespace gp {
namespace ff {

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, f2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ float2 swap(float2 a) { return f2(a.y, a.x); }

// complex float-float value; per lane value = hi + lo
struct C {
    float2 hi, lo;
};

// Expanded complex coefficient (FfCoef): a real coefficient uses rh, rl only.
using K = FfCoef;

__device__ __forceinline__ C cz() { return C{f2(0.f, 0.f), f2(0.f, 0.f)}; }

// per lane: s + e == a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add(a, b);
    const float2 bb = sub(s, a);
    e = add(sub(a, sub(s, bb)), sub(b, bb));
}

// per lane, |a| >= |b|: s + e == a + b exactly (Dekker)
__device__ __forceinline__ void fast_two_sum(float2 a, float2 b, float2 &s, float2 &e)
{
    s = add(a, b);
    e = sub(b, sub(s, a));
}

// normalised copy of z (lo within half an ulp of hi)
__device__ __forceinline__ C norm(C z)
{
    C r;
    fast_two_sum(z.hi, z.lo, r.hi, r.lo);
    return r;
}

// a + b and a - b
__device__ __forceinline__ C add(C a, C b)
{
    C r;
    two_sum(a.hi, b.hi, r.hi, r.lo);
    r.lo = add(r.lo, add(a.lo, b.lo));
    return r;
}
__device__ __forceinline__ C sub(C a, C b)
{
    C r;
    two_sum(a.hi, neg(b.hi), r.hi, r.lo);
    r.lo = add(r.lo, sub(a.lo, b.lo));
    return r;
}

// per lane product with a per-lane float-float factor (kh + kl): the exact
// product of the hi parts (TwoProduct) plus both cross terms
__device__ __forceinline__ C lmul(C z, float2 kh, float2 kl)
{
    C r;
    r.hi = mul(z.hi, kh);
    float2 e = fma2(z.hi, kh, neg(r.hi));
    e = fma2(z.hi, kl, e);
    r.lo = fma2(z.lo, kh, e);
    return r;
}

// z * k for a real coefficient k (expanded form)
__device__ __forceinline__ C rmul(C z, const K &k) { return lmul(z, k.rh, k.rl); }

// z * k for a complex coefficient k (expanded form)
__device__ __forceinline__ C cmul(C z, const K &k)
{
    const C a = lmul(z, k.rh, k.rl);
    const C b = lmul(C{swap(z.hi), swap(z.lo)}, k.ih, k.il);
    C r;
    two_sum(a.hi, b.hi, r.hi, r.lo);
    r.lo = add(r.lo, add(a.lo, b.lo));
    return r;
}

// i k z for a real k given as (kh, kl): (-k z_im, k z_re)
__device__ __forceinline__ C imul(C z, float2 kk_hi, float2 kk_lo)
{
    return lmul(C{swap(z.hi), swap(z.lo)}, kk_hi, kk_lo);
}

// 2 v - p, normalised
__device__ __forceinline__ C twice_minus(C v, C p)
{
    const float2 two = f2(2.f, 2.f);
    return norm(sub(C{mul(two, v.hi), mul(two, v.lo)}, p));
}

// |z|^2 summed over the two lanes, as a scalar float-float (hi, lo)
__device__ __forceinline__ float2 abs2(C z)
{
    const float2 p = mul(z.hi, z.hi);
    float2 e = fma2(z.hi, z.hi, neg(p));
    e = fma2(z.hi, z.lo, e);
    e = fma2(z.hi, z.lo, e);
    // scalar TwoSum of the two lanes
    const float s = p.x + p.y;
    const float bb = s - p.x;
    const float t = (p.x - (s - bb)) + (p.y - bb);
    return f2(s, t + (e.x + e.y));
}

// ---- scalar float-float helpers (per-line set-up and rare paths) ----------

__device__ __forceinline__ float2 s_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return f2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 s_norm(float2 a)
{
    const float s = a.x + a.y;
    return f2(s, a.y - (s - a.x));
}
// (a.x + a.y)(b.x + b.y), unnormalised
__device__ __forceinline__ float2 s_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return f2(p, e);
}
__device__ __forceinline__ float2 s_add(float2 a, float2 b)
{
    const float2 s = s_two_sum(a.x, b.x);
    return f2(s.x, s.y + (a.y + b.y));
}

// FP64 value as a normalised float-float pair, and back
__device__ __forceinline__ float2 split(double v)
{
    const float h = (float)v;
    return f2(h, (float)(v - (double)h));
}
__device__ __forceinline__ double join(float2 v) { return (double)v.x + (double)v.y; }

// expanded coefficient from FP64 parts
__device__ __forceinline__ K expand(double re, double im)
{
    const float2 r = split(re), i = split(im);
    return K{f2(r.x, r.x), f2(r.y, r.y), f2(-i.x, i.x), f2(-i.y, i.y)};
}

}  // namespace ff
}  // namespace gp
