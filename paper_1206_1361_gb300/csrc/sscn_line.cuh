// sscn_line.cuh -- per-point arithmetic shared by the sweep kernels: the
// Crank-Nicolson line update (calclux / calcluy / calcluz) and the
// potential / nonlinearity factor (calcnu).
#pragma once

#include "sscn_coef.cuh"
#include "sscn_internal.h"

using gp::StepG;

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

template <typename T> __device__ __forceinline__ typename Cx<T>::t cx(T x, T y)
{
    typename Cx<T>::t r;
    r.x = x;
    r.y = y;
    return r;
}

// d - v f (real coefficient)
__device__ __forceinline__ double fms_re(double d, double v, double2 f) { return fma(-f.x, v, d); }
__device__ __forceinline__ float fms_re(float d, float v, float4 f)
{
    return fmaf(-f.x, v, fmaf(-f.z, v, d));
}
// d - v f (complex coefficient)
__device__ __forceinline__ double2 fms_c(double2 d, double2 v, double2 f)
{
    return make_double2(fma(-f.x, v.x, fma(f.y, v.y, d.x)), fma(-f.x, v.y, fma(-f.y, v.x, d.y)));
}
__device__ __forceinline__ float2 fms_c(float2 d, float2 v, float4 f)
{
    const float lx = fmaf(-f.z, v.x, fmaf(f.w, v.y, d.x)), ly = fmaf(-f.z, v.y, fmaf(-f.w, v.x, d.y));
    return make_float2(fmaf(-f.x, v.x, fmaf(f.y, v.y, lx)), fmaf(-f.x, v.y, fmaf(-f.y, v.x, ly)));
}

// Crank-Nicolson line arithmetic.  MODE 0 (imaginary time): kappa = k real,
// coefficient tables real.  MODE 1 (real time): kappa = i k, tables complex.
// HI (complex64 only): apply the hi part of each FP32 hi + lo coefficient.
template <typename T, int MODE, bool HI = false> struct LineOps {
    using C = typename Cx<T>::t;
    using F = typename Coef<T>::t;
    T k;

    static __device__ __forceinline__ T rmul(T v, F f)
    {
        if constexpr (HI && sizeof(T) == 4) return rmulc_hi(v, f);
        else return rmulc(v, f);
    }
    static __device__ __forceinline__ C cmul(C v, F f)
    {
        if constexpr (HI && sizeof(T) == 4) return cmulc_hi(v, f);
        else return cmulc(v, f);
    }

    // right-hand side (1 - 2 kappa) m + kappa (l + r)
    __device__ __forceinline__ C rhs(C l, C m, C r) const
    {
        if (MODE == 0) {
            const T a = (T)1 - (T)2 * k;
            return cx<T>(fma(k, l.x + r.x, a * m.x), fma(k, l.y + r.y, a * m.y));
        }
        // (1 - 2 i k) m + i k (l + r) = m + i k (l + r - 2 m)
        const T sx = l.x + r.x - (T)2 * m.x, sy = l.y + r.y - (T)2 * m.y;
        return cx<T>(fma(-k, sy, m.x), fma(k, sx, m.y));
    }
    // forward elimination step (p + kappa d) f
    __device__ __forceinline__ C fwd(C p, C d, F f) const
    {
        if (MODE == 0) return cx<T>(rmul(fma(k, d.x, p.x), f), rmul(fma(k, d.y, p.y), f));
        return cmul(cx<T>(fma(-k, d.y, p.x), fma(k, d.x, p.y)), f);
    }
    // back substitution step d - c v
    __device__ __forceinline__ C back(C d, F c, C v) const
    {
        if constexpr (HI && sizeof(T) == 4) {
            if (MODE == 0) return cx<T>(fmaf(-c.x, v.x, d.x), fmaf(-c.x, v.y, d.y));
            return cx<T>(fmaf(-c.x, v.x, fmaf(c.y, v.y, d.x)), fmaf(-c.x, v.y, fmaf(-c.y, v.x, d.y)));
        } else {
            if (MODE == 0) return cx<T>(fms_re(d.x, v.x, c), fms_re(d.y, v.y, c));
            return fms_c(d, v, c);
        }
    }
    // u = 2 v - p  (the update when the line solves (I - kappa L) v = p)
    static __device__ __forceinline__ C out(C v, C p)
    {
        return cx<T>(fma((T)2, v.x, -p.x), fma((T)2, v.y, -p.y));
    }

    // Increment form: (I - kappa L) D = kappa L p, u = p + 2 D.  The same
    // update as u = 2 v - p (v = D + p); the recurrences carry only the
    // small D, so the one rounding left at full size is the final store.
    // kappa (l + r - 2 m):
    __device__ __forceinline__ C lap(C l, C m, C r) const
    {
        const T sx = l.x + r.x - (T)2 * m.x, sy = l.y + r.y - (T)2 * m.y;
        if (MODE == 0) return cx<T>(k * sx, k * sy);
        return cx<T>(-k * sy, k * sx);
    }
    static __device__ __forceinline__ C out_inc(C dlt, C p)
    {
        return cx<T>(fma((T)2, dlt.x, p.x), fma((T)2, dlt.y, p.y));
    }
};

// exp(-a) and exp(-i a) for the nonlinear phase a = dt g |psi|^2.
// FP64: Taylor polynomials whose degree follows |a| (read from the exponent
// bits, so the test costs no FP64 instruction), each truncated where the
// first dropped term is below 2^-54 of the result:
//   |a| <  2^-13: exp(-a) to a^3, cos to a^2, sin to a^3
//   |a| <  2^-8 : exp(-a) to a^5, cos to a^4, sin to a^5
//   |a| <= 1/16 : exp(-a) to a^9, cos to a^8, sin to a^9 (truncation < 3e-19)
// and the library function beyond.  In the usual regimes |a| stays below
// 2^-8 everywhere (dt g max|psi|^2 ~ 1e-3), and below 2^-13 outside the
// condensate's core.  FP32, real time: the update is v + delta v with delta =
// exp(-i a) - 1 formed as small numbers (cos a - 1 = -2 sin^2(a/2)), so the
// modulus of the factor carries no FP32 rounding of 1.
__device__ __forceinline__ int exp_hi(double a) { return __double2hiint(a) & 0x7fffffff; }
constexpr int kHi2m13 = 0x3f200000;     // high word of 2^-13
constexpr int kHi2m8 = 0x3f700000;      // high word of 2^-8

__device__ __forceinline__ double expm_small(double a)
{
    const int e = exp_hi(a);
    if (e < kHi2m13) return fma(fma(fma(-1.0 / 6, a, 0.5), a, -1.0), a, 1.0);
    if (e < kHi2m8) {
        double r = fma(-1.0 / 120, a, 1.0 / 24);
        r = fma(r, a, -1.0 / 6);
        r = fma(r, a, 0.5);
        r = fma(r, a, -1.0);
        return fma(r, a, 1.0);
    }
    if (fabs(a) <= 0.0625) {
        double r = -1.0 / 362880;
        r = fma(r, a, 1.0 / 40320);
        r = fma(r, a, -1.0 / 5040);
        r = fma(r, a, 1.0 / 720);
        r = fma(r, a, -1.0 / 120);
        r = fma(r, a, 1.0 / 24);
        r = fma(r, a, -1.0 / 6);
        r = fma(r, a, 0.5);
        r = fma(r, a, -1.0);
        return fma(r, a, 1.0);
    }
    return exp(-a);
}
__device__ __forceinline__ float expm_small(float a) { return expf(-a); }

__device__ __forceinline__ void expmi_small(double a, double &c, double &s)
{
    const int e = exp_hi(a);
    const double t = a * a;
    if (e < kHi2m13) {
        c = fma(t, -0.5, 1.0);
        s = a * fma(t, -1.0 / 6, 1.0);
    } else if (e < kHi2m8) {
        c = fma(t, fma(t, 1.0 / 24, -0.5), 1.0);
        s = a * fma(t, fma(t, 1.0 / 120, -1.0 / 6), 1.0);
    } else if (fabs(a) <= 0.0625) {
        c = fma(t, fma(t, fma(t, fma(t, 1.0 / 40320, -1.0 / 720), 1.0 / 24), -0.5), 1.0);
        s = a * fma(t, fma(t, fma(t, fma(t, 1.0 / 362880, -1.0 / 5040), 1.0 / 120), -1.0 / 6), 1.0);
    } else {
        sincos(a, &s, &c);
    }
}

// cos a - 1 and sin a for the update psi + (cos a - 1) psi - i sin a psi:
// both to within 2^-25 absolute, below the FP32 rounding of the result.  For
// |a| <= 1/16 the first dropped terms, a^6 / 720 and a^5 / 120, are below
// 1e-10 and 8e-9.
__device__ __forceinline__ void phase_delta(float a, float &cm1, float &s)
{
    if (fabsf(a) <= 0.0625f) {
        const float t = a * a;
        cm1 = t * fmaf(t, 1.0f / 24, -0.5f);
        s = a * fmaf(t, -1.0f / 6, 1.0f);
    } else {
        float sh, ch;
        sincosf(0.5f * a, &sh, &ch);
        cm1 = -2.0f * sh * sh;
        s = 2.0f * sh * ch;
    }
}

// calcnu at one point of a line (written for an x line; any axis works with
// the tables passed in that order): imaginary time s P exp(-dt g |s psi|^2)
// psi (P real), real time P exp(-i dt g |psi|^2) psi (P unit complex), with
// P = P_x[i] P_y[j] P_z[k] from per-axis factor tables (V is separable).
// Complex64 real time instead forms the whole phase Theta = theta_x[i] +
// theta_y[j] + theta_z[k] + dt g |psi|^2 (theta_k = dt omega_k^2 x^2 / 2, FP32
// tables) and applies psi + (exp(-i Theta) - 1) psi: one full-size rounding
// per point and a factor whose modulus carries no rounding of 1.
template <typename T, int MODE> struct Calcnu {
    using C = typename Cx<T>::t;
    using F = typename Coef<T>::t;
    const F *px;
    F pyz;          // P_y[j] P_z[k] (times the pending scale s in imaginary time)
    T a_coef;       // dt g (times s^2 in imaginary time)
    const float *tx;    // complex64 real time: theta_x table
    float tyz;          // theta_y[j] + theta_z[k]

    static __device__ __forceinline__ double2 as_d(double2 f) { return f; }
    static __device__ __forceinline__ double2 as_d(float4 f)
    {
        return make_double2((double)f.x + (double)f.z, (double)f.y + (double)f.w);
    }
    static __device__ __forceinline__ void to_f(double2 v, double2 &f) { f = v; }
    static __device__ __forceinline__ void to_f(double2 v, float4 &f)
    {
        const float hx = (float)v.x, hy = (float)v.y;
        f = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }

    // per line (j, k): factor tables (px along the line, py[j] and pz[k] for
    // the line), phase tables likewise, G (dt g for a whole step at constant
    // g), pending scale (nullptr: none)
    __device__ __forceinline__ void setup(const F *px_, const F *py, const F *pz, const float *tx_,
                                          const float *ty, const float *tz, int j, int k,
                                          double dtg, const double *scale)
    {
        px = px_;
        tx = tx_;
        const double2 y = as_d(py[j]), z = as_d(pz[k]);
        if (MODE == 0) {
            const double sc = scale ? *scale : 1.0;
            to_f(make_double2(sc * y.x * z.x, 0.0), pyz);
            a_coef = (T)(dtg * sc * sc);
            tyz = 0.f;
        } else {
            to_f(make_double2(y.x * z.x - y.y * z.y, y.x * z.y + y.y * z.x), pyz);
            a_coef = (T)dtg;
            tyz = sizeof(T) == 4 ? ty[j] + tz[k] : 0.f;
        }
    }

    __device__ __forceinline__ C apply(C v, int i) const
    {
        const T a = a_coef * fma(v.x, v.x, v.y * v.y);
        if (MODE == 0) {
            const T f = rmulc(rmulc(expm_small(a), pyz), px[i]);
            return cx<T>(v.x * f, v.y * f);
        }
        if constexpr (sizeof(T) == 8) {
            T cs, sn;
            expmi_small(a, cs, sn);
            const C w = cx<T>(fma(cs, v.x, sn * v.y), fma(cs, v.y, -sn * v.x));
            return cmulc(cmulc(w, pyz), px[i]);
        } else {
            T cm1, sn;
            phase_delta(tx[i] + tyz + a, cm1, sn);
            return cx<T>(fmaf(cm1, v.x, fmaf(sn, v.y, v.x)), fmaf(cm1, v.y, fmaf(-sn, v.x, v.y)));
        }
    }
};
