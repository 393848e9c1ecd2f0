// sscn_kernels.cu -- CUDA kernels of the split-step Crank-Nicolson step for
// sm_103a: the fused calcnu + x sweep, the y / z sweeps (calclux, calcluy,
// calcluz), the norm reduction (calcnorm) and the observables pass
// (calcmuen, calcrms) of the paper's "Summary of revisions".
//
// Every sweep runs one grid line per thread.  For the y and z sweeps the
// threads of a warp own neighbouring x, so each load and store of a point is a
// contiguous warp-wide access; the x sweep walks contiguous lines per thread
// and leans on L1.  The Thomas elimination is exact: forward elimination
// writes d'_i to a scratch buffer laid out like psi, back substitution reads
// it back in reverse.
//
// Reductions (norm partials, observables) accumulate in FP64 in a fixed order:
// per thread sequentially, then a warp-shuffle tree, then per block, so a
// given launch shape always produces the same bits (the observables do not
// depend on the launch shape at all: one partials row per grid line).

#include <cstdint>
#include <cuda_runtime.h>

#include "sscn_accum.cuh"
#include "sscn_internal.h"
#include "sscn_line.cuh"

namespace gp {
namespace {

// ------------------------------------------------------------- complex types

template <typename T> struct CT;
template <> struct CT<double> { using c = double2; };
template <> struct CT<float> { using c = float2; };

template <typename T> __device__ __forceinline__ typename CT<T>::c mk(T x, T y)
{
    typename CT<T>::c r;
    r.x = x;
    r.y = y;
    return r;
}

template <typename T> __device__ __forceinline__ T abs2(typename CT<T>::c v)
{
    return v.x * v.x + v.y * v.y;
}

template <typename T> __device__ __forceinline__ double abs2d(typename CT<T>::c v)
{
    double x = (double)v.x, y = (double)v.y;
    return x * x + y * y;
}

// ---------------------------------------------------------- block reduction

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum v over the block in a fixed order; the result is valid in thread 0.
__device__ double block_sum(double v, double *red /* >= 32 doubles */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();                       // red may be reused by the caller
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < nwarps ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// ------------------------------------------------------------------ sweeps
//
// Each Crank-Nicolson line update (I - kappa L) u = (I + kappa L) psi is done
// as u = 2 v - psi with (I - kappa L) v = psi, using I + kappa L =
// 2 I - (I - kappa L): the same solution without forming the right-hand side
// stencil, which saves a third of the FP64 instructions per point (the FP64
// pipe bounds these kernels on GB300).  Forward elimination:
// d'_i = (psi_i + kappa d'_{i-1}) mult_i into the scratch buffer; back
// substitution: v_i = d'_i - c'_i v_{i+1}, u_i = 2 v_i - psi_i.

// Two-ended elimination ("burn at both ends", a twisted factorisation): the
// lane pair (l, l ^ 16) of a warp owns one line; the low lane eliminates from
// the top (i = 1 .. k-1), the high lane from the bottom (i = m .. k+1) with the
// mirrored tables (the matrix is symmetric Toeplitz, so the reversed system
// has the same coefficients), they meet at the middle unknown k =
// ceil(m / 2), and back-substitute outward.  Same FP64 work as one-sided
// Thomas, twice the independent chains: 16 lines per warp.
//   top:    d'_i = (psi_i + kappa d'_{i-1}) mult_i,      v_i = d'_i - c'_i v_{i+1}
//   bottom: e_i  = (psi_i + kappa e_{i+1}) mult_{m+1-i}, v_i = e_i - c'_{m+1-i} v_{i-1}
//   middle: v_k  = (psi_k + kappa (d'_{k-1} + e_{k+1})) mid,
//           mid  = 1 / (1 + 2 kappa + kappa (c'_{k-1} + c'_{m-k})), c'_0 = 0.
#ifndef GP_SWEEP_THREADS
#define GP_SWEEP_THREADS 64
#endif
constexpr int kSweepThreads = GP_SWEEP_THREADS;
#ifndef GP_SWEEP_PREFETCH
#define GP_SWEEP_PREFETCH 4
#endif
constexpr int kPrefetch = GP_SWEEP_PREFETCH;     // points loaded ahead per thread
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ typename CT<T>::c shfl_xor16(typename CT<T>::c v)
{
    v.x = __shfl_xor_sync(kFull, v.x, 16);
    v.y = __shfl_xor_sync(kFull, v.y, 16);
    return v;
}

// NL: calcnu on each point as it is loaded (the x sweep); NLOUT: calcnu on
// each result before it is stored (the second half step of the symmetric
// splitting, in the last sweep).  P3 (FP64 real time): the potential factor
// P_x[i] P_y[j] P_z[k] of each point comes from a precomputed table laid out
// like psi (one complex multiply per point instead of two; 16 more bytes read
// per point by a sweep that is bound by the FP64 pipe, not by HBM).
template <typename T, int MODE, bool NL, bool NORM, bool NLOUT = false, bool P3 = false>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep(typename CT<T>::c *__restrict__ psi, typename CT<T>::c *__restrict__ work,
        const typename Coef<T>::t *__restrict__ cp,
        const typename Coef<T>::t *__restrict__ mult, typename Coef<T>::t mid, SweepGeom g,
        T kappa, const typename Coef<T>::t *__restrict__ px,
        const typename Coef<T>::t *__restrict__ py, const typename Coef<T>::t *__restrict__ pz,
        const float *__restrict__ tx, const float *__restrict__ ty, const float *__restrict__ tz,
        StepG sg, const double *__restrict__ scale, double *__restrict__ partials,
        const double *__restrict__ lw, const double2 *__restrict__ p3)
{
    using C = typename CT<T>::c;
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    const bool top = lane < 16;
    const int a = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16 + (lane & 15);
    const int b = blockIdx.y;
    const bool active = a < g.lines_a;
    const int m = g.n - 1;
    const int k = (m + 1) >> 1;              // middle unknown
    const int len = top ? k - 1 : m - k;     // points this lane eliminates
    const long long s = g.pstride;
    const long long base = active ? (long long)a * g.stride_a + (long long)b * g.stride_b : 0;
    C *line = psi + base;
    C *wl = work + base;
    const LineOps<T, MODE> cn{kappa};
    Calcnu<T, MODE> nl{};
    if ((NL || NLOUT) && active && !P3) nl.setup(px, py, pz, tx, ty, tz, a, b, sg.value(), scale);
    const double G3 = P3 ? sg.value() : 0.0;
    const double2 *p3l = p3 + (P3 ? base : 0);
    // calcnu at stored point i of this line
    auto calcnu = [&](C v, int i) -> C {
        if constexpr (P3 && sizeof(T) == 8 && MODE == 1) {
            double cs, sn;
            expmi_small(G3 * fma(v.x, v.x, v.y * v.y), cs, sn);
            const double2 w = make_double2(fma(cs, v.x, sn * v.y), fma(cs, v.y, -sn * v.x));
            return cmulc(w, p3l[(long long)i * s]);
        } else {
            return nl.apply(v, i);
        }
    };
    Acc<T> nacc;
    C d = mk<T>((T)0, (T)0);
    if (active) {
        // loads are issued kPrefetch points at a time, ahead of the
        // recurrence that consumes them
        for (int t0 = 0; t0 < len; t0 += kPrefetch) {
            C pv[kPrefetch];
#pragma unroll
            for (int q = 0; q < kPrefetch; ++q)
                if (t0 + q < len) pv[q] = line[(long long)(top ? 1 + t0 + q : m - t0 - q) * s];
#pragma unroll
            for (int q = 0; q < kPrefetch; ++q) {
                const int t = t0 + q;
                if (t < len) {
                    const int i = top ? 1 + t : m - t;
                    const long long at = (long long)i * s;
                    C p = pv[q];
                    if (NL) {
                        p = calcnu(p, i);
                        line[at] = p;
                    }
                    d = cn.fwd(p, d, mult[t]);
                    wl[at] = d;
                }
            }
        }
    }
    const C other = shfl_xor16<T>(d);
    C vk = mk<T>((T)0, (T)0);
    if (active && top) {
        C pk = line[(long long)k * s];
        if (NL) pk = calcnu(pk, k);
        vk = cn.fwd(pk, mk<T>(d.x + other.x, d.y + other.y), mid);
        C u = LineOps<T, MODE>::out(vk, pk);
        if (NLOUT) u = calcnu(u, k);
        line[(long long)k * s] = u;
        if (NORM) nacc.add(abs2<T>(u));
    }
    const C vpair = shfl_xor16<T>(vk);
    C v = top ? vk : vpair;
    if (active) {
        for (int t0 = len - 1; t0 >= 0; t0 -= kPrefetch) {
            C wv[kPrefetch], lv[kPrefetch];
#pragma unroll
            for (int q = 0; q < kPrefetch; ++q)
                if (t0 - q >= 0) {
                    const long long at = (long long)(top ? 1 + t0 - q : m - t0 + q) * s;
                    wv[q] = wl[at];
                    lv[q] = line[at];
                }
#pragma unroll
            for (int q = 0; q < kPrefetch; ++q) {
                const int t = t0 - q;
                if (t >= 0) {
                    const long long at = (long long)(top ? 1 + t : m - t) * s;
                    v = cn.back(wv[q], cp[t], v);
                    C u = LineOps<T, MODE>::out(v, lv[q]);
                    if (NLOUT) u = calcnu(u, top ? 1 + t : m - t);
                    line[at] = u;
                    if (NORM) nacc.add(abs2<T>(u));
                }
            }
        }
    }
    if (NORM) {
        double part = nacc.get();
        if (lw && active) part *= lw[a];
        const double r = block_sum(part, red);
        if (threadIdx.x == 0) partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = r;
    }
}

constexpr int kLinesPerBlock = kSweepThreads / 2;

template <typename T, int MODE, bool NL, bool NORM, bool NLOUT = false, bool P3 = false>
cudaError_t sweep_launch(void *psi, void *work, const AxisTables &ax,
                         const SweepGeom &g, const NonlinArgs *nl,
                         const Partials *norm_out, cudaStream_t st)
{
    using C = typename CT<T>::c;
    using F = typename Coef<T>::t;
    dim3 grid((g.lines_a + kLinesPerBlock - 1) / kLinesPerBlock, g.lines_b);
    const F *cp, *mult, *px = nullptr, *py = nullptr, *pz = nullptr;
    const float *tx = nl ? nl->tx32 : nullptr, *ty = nl ? nl->ty32 : nullptr, *tz = nl ? nl->tz32 : nullptr;
    F mid;
    T kappa = (T)(MODE == 0 ? ax.kre : ax.kim);
    if constexpr (sizeof(T) == 8) {
        cp = ax.cp64;
        mult = ax.mult64;
        mid = ax.mid64;
        if (nl) { px = nl->px; py = nl->py; pz = nl->pz; }
    } else {
        cp = ax.cp32;
        mult = ax.mult32;
        mid = ax.mid32;
        if (nl) { px = nl->px32; py = nl->py32; pz = nl->pz32; }
    }
    k_sweep<T, MODE, NL, NORM, NLOUT, P3><<<grid, kSweepThreads, 0, st>>>(
        reinterpret_cast<C *>(psi), reinterpret_cast<C *>(work), cp, mult, mid, g, kappa,
        px, py, pz, tx, ty, tz, nl ? nl->g : StepG{}, nl ? nl->scale : nullptr,
        norm_out ? norm_out->buf : nullptr, norm_out ? norm_out->line_weight : nullptr,
        nl ? nl->p3 : nullptr);
    return cudaGetLastError();
}

template <typename T, bool NL>
cudaError_t sweep_dispatch(int mode, void *psi, void *work, const AxisTables &ax,
                           const SweepGeom &g, const NonlinArgs *nl,
                           const Partials *norm_out, cudaStream_t st)
{
    if (mode == 0) {
        if (norm_out) return sweep_launch<T, 0, NL, true>(psi, work, ax, g, nl, norm_out, st);
        return sweep_launch<T, 0, NL, false>(psi, work, ax, g, nl, norm_out, st);
    }
    if (norm_out) return sweep_launch<T, 1, NL, true>(psi, work, ax, g, nl, norm_out, st);
    return sweep_launch<T, 1, NL, false>(psi, work, ax, g, nl, norm_out, st);
}

// ------------------------------------------------------- pointwise kernels

__global__ void k_norm_finish(const double *__restrict__ partials, int count,
                              double w, double *scale, double *norm_out, int *err)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += partials[i];
    const double total = block_sum(v, red);
    if (threadIdx.x == 0) {
        const double n = w * total;
        if (norm_out) *norm_out = n;
        if (!(n > 0.0) || !isfinite(n)) {
            atomicOr(err, 1);
            *scale = 1.0;
        } else {
            *scale = 1.0 / sqrt(n);
        }
    }
}

template <typename T>
__global__ void k_apply_scale(typename CT<T>::c *__restrict__ psi, long long count,
                              const double *__restrict__ scale)
{
    const T s = (T)(*scale);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        auto v = psi[p];
        v.x *= s;
        v.y *= s;
        psi[p] = v;
    }
}

__global__ void k_set_one(double *x) { *x = 1.0; }

__device__ __forceinline__ double coord(int n, double h, int i)
{
    return n == 1 ? 0.0 : -0.5 * (double)n * h + (double)i * h;
}

template <typename T>
__global__ void k_seed(typename CT<T>::c *__restrict__ psi, int nx, int ny, int nz,
                       double hx, double hy, double hz, double gx, double gy, double gz)
{
    const long long count = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx);
        const int j = (int)((p / nx) % ny);
        const int k = (int)(p / ((long long)nx * ny));
        const bool edge = i == 0 || j == 0 || (nz > 1 && k == 0);
        double v = 0.0;
        if (!edge) {
            const double x = coord(nx, hx, i), y = coord(ny, hy, j), z = coord(nz, hz, k);
            v = exp(-0.5 * (gx * x * x + gy * y * y + gz * z * z));
        }
        psi[p] = mk<T>((T)v, (T)0);
    }
}

template <typename T>
__global__ void k_zero_boundary(typename CT<T>::c *__restrict__ psi, int nx, int ny, int nz)
{
    const long long count = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx);
        const int j = (int)((p / nx) % ny);
        const int k = (int)(p / ((long long)nx * ny));
        if (i == 0 || j == 0 || (nz > 1 && k == 0)) psi[p] = mk<T>((T)0, (T)0);
    }
}

template <typename T>
__global__ void k_norm_partials(const typename CT<T>::c *__restrict__ psi, long long count,
                                double *__restrict__ partials)
{
    __shared__ double red[32];
    double v = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x)
        v += abs2d<T>(psi[p]);
    const double r = block_sum(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// calcnu as a pass of its own: one warp per x line (j, k), fixed line-to-warp
// assignment, FP64 sum |u|^2 per block (imaginary-time symmetric splitting:
// the second half step after the renormalisation, with the pending scale).
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
k_calcnu_pass(typename CT<T>::c *__restrict__ psi, int nx, int ny, int nz,
              const typename Coef<T>::t *__restrict__ px, const typename Coef<T>::t *__restrict__ py,
              const typename Coef<T>::t *__restrict__ pz, const float *__restrict__ tx,
              const float *__restrict__ ty, const float *__restrict__ tz, StepG sg,
              const double *__restrict__ scale, double *__restrict__ partials,
              const double *__restrict__ wx)
{
    using C = typename CT<T>::c;
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const double G = sg.value();
    const long long lines = (long long)ny * nz;
    double acc = 0.0;
    for (long long L = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); L < lines;
         L += warps) {
        const int j = (int)(L % ny), k = (int)(L / ny);
        Calcnu<T, MODE> nl{};
        nl.setup(px, py, pz, tx, ty, tz, j, k, G, scale);
        C *line = psi + L * nx;
        for (int i = lane; i < nx; i += 32) {
            const C u = nl.apply(line[i], i);
            line[i] = u;
            acc = fma(wx ? wx[i] : 1.0, abs2d<T>(u), acc);
        }
    }
    const double r = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// The potential factor table P[(k ny + j) nx + i] = P_x[i] P_y[j] P_z[k].
__global__ void k_build_pot3(double2 *__restrict__ p3, const double2 *__restrict__ px,
                             const double2 *__restrict__ py, const double2 *__restrict__ pz,
                             int nx, int ny, int nz)
{
    const long long count = (long long)nx * ny * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((long long)nx * ny));
        p3[p] = cmulc(cmulc(py[j], pz[k]), px[i]);
    }
}

__global__ void k_set_step(long long *step, long long value) { *step = value; }
__global__ void k_add_step(long long *step) { *step += 1; }

// ------------------------------------------------------------ observables
//
// Per x-line (j, k), FP64 grids: one thread walks the line in order
// (consecutive threads on consecutive lines; the line's points come through
// L1).  Per point: a = |psi|^2, its x^2 and V_x weighted sums, |psi|^4, and the
// neighbour terms along x, y and z (zero beyond the last stored point); the
// y and z coordinate factors are constant on the line, so sum y^2 |psi|^2 =
// y_j^2 sum |psi|^2 etc. are formed once per line.  Each line writes its 9
// sums (times the pending scale s^2, s^4 for |psi|^4) to its own partials
// row; two fixed-order passes add the rows, so the result does not depend on
// the launch shape.  A thread per line keeps every sum in one thread: no
// warp reduction per line, which on GB300 (2 FP64 FMA per clock per SM) cost
// more than the points themselves.
//
// FP64: the neighbour terms are R_k = sum Re(psi_next conj(psi)) (2 FMA),
// and the finish forms K_k = 2 S0 - 2 R_k (every point is once "next" and
// once "current", the boundary values are zero): sum |psi_next - psi|^2
// exactly, with a relative rounding of ~1e-14 after the cancellation.
//
// complex64 (FP32 terms, memory-bound) keeps a warp per line for coalesced
// loads and the differences (the cancellation would amplify FP32 rounding past
// the 1e-6 the form is held to); its lanes' compensated FP32 partials are
// combined across the warp in FP32 with an error-free sum (TwoSum), not in
// FP64, and lane 0 converts the line's totals.

constexpr int kObsThreads = 256;
constexpr int kObsChunk = 1024;          // lines per first-stage finish block

// A thread owns one x and walks a chunk of kObsLines consecutive y-lines of
// one plane (blocks over x segments, line chunks and planes): each point is
// loaded once as the thread's own value and carried to the next line as that
// line's y-neighbour; the x-neighbour comes from the next lane (lane 31 loads
// it), the z-neighbour from the next plane, which the blocks of that plane
// (resident at the same time) find in L2.  The factors constant for the
// thread (x^2, V_x) or the block (z^2, V_z) multiply its partial of |psi|^2
// once; those of a line (y^2, V_y) are staged in shared memory per block.
// Each block writes one row of 9 sums.
__global__ void __launch_bounds__(256)
k_observables_c64(const float2 *__restrict__ psi, ObsArgs a, double *__restrict__ rows)
{
    __shared__ float yt[2][kObsLines];
    __shared__ double red[8][9];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = blockIdx.y * kObsLines, j1 = min(j0 + kObsLines, ny);
    const int k = blockIdx.z;
    for (int t = threadIdx.x; t < kObsLines && j0 + t < ny; t += blockDim.x) {
        yt[0][t] = (float)a.y2[j0 + t];
        yt[1][t] = (float)a.vy[j0 + t];
    }
    __syncthreads();
    const bool in = i < nx, has_z = k + 1 < nz;
    const long long plane = (long long)nx * ny;
    const float2 *pk = psi + k * plane;
    const float2 zero = make_float2(0.f, 0.f);
    Acc<float> s0, sy, svy, s4, kx, ky, kz;
    float2 v = in ? pk[(long long)j0 * nx + i] : zero;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const long long at = (long long)j * nx + i;
        const float2 vn = (in && j + 1 < ny) ? pk[at + nx] : zero;      // y-neighbour
        const float2 vz = (in && has_z) ? pk[at + plane] : zero;         // z-neighbour
        float2 nb;                                                       // x-neighbour
        nb.x = __shfl_down_sync(0xffffffffu, v.x, 1);
        nb.y = __shfl_down_sync(0xffffffffu, v.y, 1);
        if (lane == 31) nb = (i + 1 < nx) ? pk[at + 1] : zero;
        const float am = fmaf(v.x, v.x, v.y * v.y);
        s0.add(am);
        sy.add(yt[0][j - j0] * am);
        svy.add(yt[1][j - j0] * am);
        s4.add(am * am);
        kx.add_sq2(nb.x - v.x, nb.y - v.y);
        ky.add_sq2(vn.x - v.x, vn.y - v.y);
        if (nz > 1) kz.add_sq2(vz.x - v.x, vz.y - v.y);
        v = vn;
    }
    const float p0 = s0.s - s0.c;
    const float x2 = in ? a.x2f[i] : 0.f, vx = in ? a.vxf[i] : 0.f;
    // S0, Sx, Sy, SVx + SVy, S4, Kx, Ky, Kz
    const float ps[8][2] = {{s0.s, s0.c}, {x2 * p0, 0.f}, {sy.s, sy.c}, {vx * p0 + (svy.s - svy.c), 0.f},
                            {s4.s, s4.c}, {kx.s, kx.c}, {ky.s, ky.c}, {kz.s, kz.c}};
    double r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = warp_sum_comp(ps[q][0], ps[q][1]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[wib][q] = r[q];
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sc = *a.scale, s2 = sc * sc;
        const double *t = red[0];
        double *out = rows + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x * kObsWidth +
                      (long long)blockIdx.x * kObsWidth;
        out[0] = s2 * t[0];
        out[1] = s2 * t[1];
        out[2] = s2 * t[2];
        out[3] = s2 * a.z2[k] * t[0];
        out[4] = s2 * (t[3] + a.vz[k] * t[0]);
        out[5] = s2 * s2 * t[4];
        out[6] = s2 * t[5];
        out[7] = s2 * t[6];
        out[8] = s2 * t[7];
    }
}

// Thread per line (FP64 grids).
template <typename T>
__global__ void __launch_bounds__(kObsThreads)
k_observables(const typename CT<T>::c *__restrict__ psi, ObsArgs a,
              double *__restrict__ partials)
{
    using C = typename CT<T>::c;
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    if (line >= (long long)ny * nz) return;
    const int j = (int)(line % ny), k = (int)(line / ny);
    const long long plane = (long long)nx * ny;
    const C *row = psi + line * nx;
    const bool has_y = j + 1 < ny, has_z = nz > 1 && k + 1 < nz;
    const T *x2 = sizeof(T) == 8 ? (const T *)a.x2 : (const T *)a.x2f;
    const T *vx = sizeof(T) == 8 ? (const T *)a.vx : (const T *)a.vxf;
    constexpr bool RFORM = sizeof(T) == 8;
    Acc<T> s0, sx, svx, s4, kx, ky, kz;
    const C zero = mk<T>((T)0, (T)0);
    C v = row[0];
    for (int i = 0; i < nx; ++i) {
        const C nb = (i + 1 < nx) ? row[i + 1] : zero;
        const C ny_ = has_y ? row[i + nx] : zero;
        const C nz_ = has_z ? row[i + plane] : zero;
        const T am = fma(v.x, v.x, v.y * v.y);
        s0.add(am);
        sx.add_prod(x2[i], am);
        svx.add_prod(vx[i], am);
        s4.add_prod(am, am);
        if constexpr (RFORM) {
            kx.s = fma(nb.x, v.x, fma(nb.y, v.y, kx.s));
            ky.s = fma(ny_.x, v.x, fma(ny_.y, v.y, ky.s));
            kz.s = fma(nz_.x, v.x, fma(nz_.y, v.y, kz.s));
        } else {
            kx.add_sq2(nb.x - v.x, nb.y - v.y);
            ky.add_sq2(ny_.x - v.x, ny_.y - v.y);
            if (nz > 1) kz.add_sq2(nz_.x - v.x, nz_.y - v.y);
        }
        v = nb;
    }
    const double sc = *a.scale, s2 = sc * sc;
    const double r0 = s0.get();
    double *out = partials + line * kObsWidth;
    out[0] = s2 * r0;
    out[1] = s2 * sx.get();
    out[2] = s2 * a.y2[j] * r0;
    out[3] = s2 * a.z2[k] * r0;
    out[4] = s2 * (svx.get() + (a.vy[j] + a.vz[k]) * r0);
    out[5] = s2 * s2 * s4.get();
    out[6] = s2 * kx.get();
    out[7] = s2 * ky.get();
    out[8] = s2 * kz.get();
}

// Sum rows [b * chunk, (b + 1) * chunk) of a [rows][9] array into out[b][9].
__global__ void __launch_bounds__(256)
k_rows_sum(const double *__restrict__ rows, long long count, int chunk,
           double *__restrict__ out)
{
    __shared__ double red[32];
    const long long r0 = (long long)blockIdx.x * chunk;
    long long r1 = r0 + chunk;
    if (r1 > count) r1 = count;
    for (int q = 0; q < kObsWidth; ++q) {
        double v = 0.0;
        for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) v += rows[r * kObsWidth + q];
        const double t = block_sum(v, red);
        if (threadIdx.x == 0) out[(long long)blockIdx.x * kObsWidth + q] = t;
    }
}

constexpr int kPointThreads = 256;

int point_blocks(long long count)
{
    long long b = (count + kPointThreads - 1) / kPointThreads;
    if (b > kReduceBlocks) b = kReduceBlocks;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ================================================================ launchers

int sweep_blocks(const SweepGeom &g)
{
    return ((g.lines_a + kLinesPerBlock - 1) / kLinesPerBlock) * g.lines_b;
}

cudaError_t launch_sweep_x(int prec, int mode, void *psi, void *work,
                           const AxisTables &ax, const SweepGeom &g,
                           const NonlinArgs &nl, int, int, const Partials *norm_out,
                           cudaStream_t st)
{
    if (nl.p3) {
        // the precomputed potential factors: FP64 real time, no norm partials
        if (prec != kC128 || mode != 1 || norm_out) return cudaErrorInvalidValue;
        return sweep_launch<double, 1, true, false, false, true>(psi, work, ax, g, &nl, nullptr, st);
    }
    if (prec == kC128) return sweep_dispatch<double, true>(mode, psi, work, ax, g, &nl, norm_out, st);
    return sweep_dispatch<float, true>(mode, psi, work, ax, g, &nl, norm_out, st);
}

cudaError_t launch_sweep_yz(int prec, int mode, void *psi, void *work,
                            const AxisTables &ax, const SweepGeom &g,
                            const Partials *norm_out, cudaStream_t st, const NonlinArgs *nlout)
{
    if (nlout) {
        // the symmetric splitting's second half step, fused where the real-time
        // last sweep stores (imaginary time takes a separate pass after the
        // renormalisation)
        if (mode != 1 || norm_out) return cudaErrorInvalidValue;
        if (prec == kC128) {
            if (nlout->p3) return sweep_launch<double, 1, false, false, true, true>(psi, work, ax, g, nlout, nullptr, st);
            return sweep_launch<double, 1, false, false, true>(psi, work, ax, g, nlout, nullptr, st);
        }
        return sweep_launch<float, 1, false, false, true>(psi, work, ax, g, nlout, nullptr, st);
    }
    if (prec == kC128) return sweep_dispatch<double, false>(mode, psi, work, ax, g, nullptr, norm_out, st);
    return sweep_dispatch<float, false>(mode, psi, work, ax, g, nullptr, norm_out, st);
}

cudaError_t launch_norm_finish(const double *partials, int count, double w,
                               double *scale, double *norm_out, int *err, cudaStream_t st)
{
    k_norm_finish<<<1, 256, 0, st>>>(partials, count, w, scale, norm_out, err);
    return cudaGetLastError();
}

cudaError_t launch_apply_scale(int prec, void *psi, long long count, double *scale,
                               cudaStream_t st)
{
    const int blocks = point_blocks(count);
    if (prec == kC128)
        k_apply_scale<double><<<blocks, kPointThreads, 0, st>>>((double2 *)psi, count, scale);
    else
        k_apply_scale<float><<<blocks, kPointThreads, 0, st>>>((float2 *)psi, count, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_set_one<<<1, 1, 0, st>>>(scale);
    return cudaGetLastError();
}

cudaError_t launch_seed(int prec, void *psi, int nx, int ny, int nz, const double h[3],
                        const double w[3], cudaStream_t st)
{
    const long long count = (long long)nx * ny * nz;
    const int blocks = point_blocks(count);
    if (prec == kC128)
        k_seed<double><<<blocks, kPointThreads, 0, st>>>((double2 *)psi, nx, ny, nz, h[0], h[1], h[2], w[0], w[1], w[2]);
    else
        k_seed<float><<<blocks, kPointThreads, 0, st>>>((float2 *)psi, nx, ny, nz, h[0], h[1], h[2], w[0], w[1], w[2]);
    return cudaGetLastError();
}

cudaError_t launch_zero_boundary(int prec, void *psi, int nx, int ny, int nz, cudaStream_t st)
{
    const long long count = (long long)nx * ny * nz;
    const int blocks = point_blocks(count);
    if (prec == kC128)
        k_zero_boundary<double><<<blocks, kPointThreads, 0, st>>>((double2 *)psi, nx, ny, nz);
    else
        k_zero_boundary<float><<<blocks, kPointThreads, 0, st>>>((float2 *)psi, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_norm_partials(int prec, const void *psi, long long count,
                                 const Partials &out, int blocks, cudaStream_t st)
{
    if (prec == kC128)
        k_norm_partials<double><<<blocks, kPointThreads, 0, st>>>((const double2 *)psi, count, out.buf);
    else
        k_norm_partials<float><<<blocks, kPointThreads, 0, st>>>((const float2 *)psi, count, out.buf);
    return cudaGetLastError();
}

cudaError_t launch_calcnu_pass(int prec, int mode, void *psi, int nx, int ny, int nz,
                               const NonlinArgs &nl, const Partials &norm_out, int blocks,
                               cudaStream_t st, const double *wx)
{
    if (prec == kC128) {
        auto k = mode == 0 ? k_calcnu_pass<double, 0> : k_calcnu_pass<double, 1>;
        k<<<blocks, 256, 0, st>>>((double2 *)psi, nx, ny, nz, nl.px, nl.py, nl.pz, nl.tx32, nl.ty32,
                                  nl.tz32, nl.g, nl.scale, norm_out.buf, wx);
    } else {
        auto k = mode == 0 ? k_calcnu_pass<float, 0> : k_calcnu_pass<float, 1>;
        k<<<blocks, 256, 0, st>>>((float2 *)psi, nx, ny, nz, nl.px32, nl.py32, nl.pz32, nl.tx32,
                                  nl.ty32, nl.tz32, nl.g, nl.scale, norm_out.buf, wx);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_pot3(void *p3, const double2 *px, const double2 *py, const double2 *pz,
                              int nx, int ny, int nz, cudaStream_t st)
{
    k_build_pot3<<<4 * kReduceBlocks, 256, 0, st>>>((double2 *)p3, px, py, pz, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_set_step(long long *step, long long value, cudaStream_t st)
{
    k_set_step<<<1, 1, 0, st>>>(step, value);
    return cudaGetLastError();
}

cudaError_t launch_add_step(long long *step, cudaStream_t st)
{
    k_add_step<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

void obs_walk_geometry(int nx, int ny, int nz, dim3 &grid, int &threads)
{
    threads = 32 * ((nx + 31) / 32);
    if (threads > 256) threads = 256;
    grid = dim3((unsigned)((nx + threads - 1) / threads), (unsigned)((ny + kObsLines - 1) / kObsLines),
                (unsigned)nz);
}

long long obs_scratch_doubles(const ObsArgs &a)
{
    dim3 grid;
    int threads = 0;
    obs_walk_geometry(a.nx, a.ny, a.nz, grid, threads);
    long long rows = (long long)a.ny * a.nz;       // a row per line (FP64)
    const long long walk = (long long)grid.x * grid.y * grid.z;
    if (walk > rows) rows = walk;
    const long long chunks = (rows + kObsChunk - 1) / kObsChunk;
    return (rows + chunks) * kObsWidth;
}

cudaError_t launch_observables(int prec, const void *psi, const ObsArgs &a,
                               double *scratch, double *sums, cudaStream_t st)
{
    const long long lines = (long long)a.ny * a.nz;
    double *rows = scratch, *stage = scratch + lines * kObsWidth;
    if (prec == kC128) {
        const long long blocks = (lines + kObsThreads - 1) / kObsThreads;
        k_observables<double><<<(unsigned)blocks, kObsThreads, 0, st>>>((const double2 *)psi, a, rows);
    } else {
        dim3 grid;
        int threads = 0;
        obs_walk_geometry(a.nx, a.ny, a.nz, grid, threads);
        k_observables_c64<<<grid, threads, 0, st>>>((const float2 *)psi, a, rows);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const long long nrows = (long long)grid.x * grid.y * grid.z;
        return launch_rows_finish(rows, nrows, rows + nrows * kObsWidth, sums, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rows_finish(rows, lines, stage, sums, st);
}

cudaError_t launch_rows_finish(const double *rows, long long lines, double *stage, double *sums,
                               cudaStream_t st)
{
    const long long chunks = (lines + kObsChunk - 1) / kObsChunk;
    k_rows_sum<<<(unsigned)chunks, 256, 0, st>>>(rows, lines, kObsChunk, stage);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rows_sum<<<1, 256, 0, st>>>(stage, chunks, (int)chunks, sums);
    return cudaGetLastError();
}

}  // namespace gp
