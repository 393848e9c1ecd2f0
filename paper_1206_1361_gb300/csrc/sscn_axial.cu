// sscn_axial.cu -- the axially symmetric form psi(rho, z) (the paper's
// axially symmetric programs, summaries vii, viii, xvi, xvii): the radial
// Crank-Nicolson sweep with its non-constant coefficients and calcnu fused,
// the seed, the rho-weighted norm and the observables.  The axial sweep is
// the Cartesian y sweep of the (n_r x n_z) grid (sscn_kernels.cu).
//
// Radial grid rho_i = (i + 1/2) h_r, i = 0 .. n_r - 1, all unknowns; the
// conservative operator tridiag(a_i, -2, c_i) / h_r^2 with a_i = rho_{i-1/2} /
// rho_i = 1 - 1/(2i+1), c_i = 1 + 1/(2i+1) is self-adjoint in the
// rho-weighted inner product, so the sweep conserves 2 pi h_r h_z sum rho |psi|^2
// in real time.  Each line is eliminated from both ends by a lane pair (as
// the Cartesian sweeps do), with separate top and bottom tables because the
// coefficients are not symmetric, and the update is u = 2 v - psi with
// (I - kappa T) v = psi.

#include <cmath>
#include <complex>
#include <vector>

#include <cuda_runtime.h>

#include "sscn_accum.cuh"
#include "sscn_internal.h"
#include "sscn_line.cuh"

namespace gp {
namespace {

constexpr int kThreads = 64;                 // 2 warps, 16 lines per warp
constexpr int kLinesPerBlock = kThreads / 2;
constexpr int kPrefetchR = 4;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double2 shfl16(double2 v)
{
    v.x = __shfl_xor_sync(kFull, v.x, 16);
    v.y = __shfl_xor_sync(kFull, v.y, 16);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < nwarps ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Radial sweep of line k (z index) = psi[k * nr .. k * nr + nr - 1]; unknown
// j = 1 .. m (m = nr) sits at stored index j - 1.  Top lane: j = 1 .. kmid-1,
// bottom lane: j = m .. kmid+1, the top lane closes the middle row.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_sweep_rho(double2 *__restrict__ psi, double2 *__restrict__ work, const RadialTables rt,
            int nr, int nz, const double2 *__restrict__ pr, const double2 *__restrict__ pz,
            const double2 *__restrict__ one, StepG sg, const double *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const bool top = lane < 16;
    const int line = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16 + (lane & 15);
    const bool active = line < nz;
    const int m = nr;
    const int kmid = (m + 1) >> 1;
    const int len = top ? kmid - 1 : m - kmid;
    const long long base = active ? (long long)line * nr : 0;
    double2 *row = psi + base;
    double2 *wl = work + base;
    const double2 *cp = top ? rt.cp_top : rt.cp_bot;
    const double2 *mult = top ? rt.mult_top : rt.mult_bot;
    const double *kk = top ? rt.ka_top : rt.kc_bot;
    Calcnu<double, MODE> nl{};
    if (active) nl.setup(pr, pz, one, nullptr, nullptr, nullptr, line, 0, sg.value(), scale);
    double2 d = make_double2(0.0, 0.0);
    if (active) {
        for (int t0 = 0; t0 < len; t0 += kPrefetchR) {
            double2 pv[kPrefetchR];
#pragma unroll
            for (int q = 0; q < kPrefetchR; ++q)
                if (t0 + q < len) pv[q] = row[top ? t0 + q : m - 1 - t0 - q];
#pragma unroll
            for (int q = 0; q < kPrefetchR; ++q) {
                const int t = t0 + q;
                if (t < len) {
                    const int i = top ? t : m - 1 - t;
                    const double2 p = nl.apply(pv[q], i);
                    row[i] = p;
                    d = LineOps<double, MODE>{kk[t]}.fwd(p, d, mult[t]);
                    wl[i] = d;
                }
            }
        }
    }
    const double2 other = shfl16(d);
    double2 vk = make_double2(0.0, 0.0);
    if (active && top) {
        const int i = kmid - 1;
        const double2 pk = nl.apply(row[i], i);
        // kappa (a_k d'_{k-1} + c_k e_{k+1}) as kappa^ q with |kappa| folded into q
        const double2 q = make_double2(fma(rt.ka_mid, d.x, rt.kc_mid * other.x),
                                       fma(rt.ka_mid, d.y, rt.kc_mid * other.y));
        vk = LineOps<double, MODE>{1.0}.fwd(pk, q, rt.mid);
        row[i] = LineOps<double, MODE>::out(vk, pk);
    }
    const double2 vpair = shfl16(vk);
    double2 v = top ? vk : vpair;
    if (active) {
        for (int t0 = len - 1; t0 >= 0; t0 -= kPrefetchR) {
            double2 wv[kPrefetchR], lv[kPrefetchR];
#pragma unroll
            for (int q = 0; q < kPrefetchR; ++q)
                if (t0 - q >= 0) {
                    const int i = top ? t0 - q : m - 1 - t0 + q;
                    wv[q] = wl[i];
                    lv[q] = row[i];
                }
#pragma unroll
            for (int q = 0; q < kPrefetchR; ++q) {
                const int t = t0 - q;
                if (t >= 0) {
                    const int i = top ? t : m - 1 - t;
                    v = LineOps<double, MODE>{0.0}.back(wv[q], cp[t], v);
                    row[i] = LineOps<double, MODE>::out(v, lv[q]);
                }
            }
        }
    }
}

__global__ void k_seed_axial(double2 *__restrict__ psi, int nr, int nz, double hr, double hz,
                             double gamma, double lambda)
{
    const long long count = (long long)nr * nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nr), k = (int)(p / nr);
        double v = 0.0;
        if (k > 0) {
            const double r = (i + 0.5) * hr, z = -0.5 * nz * hz + k * hz;
            v = exp(-0.5 * (gamma * r * r + lambda * z * z));
        }
        psi[p] = make_double2(v, 0.0);
    }
}

__global__ void k_zero_axial(double2 *__restrict__ psi, int nr)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x)
        psi[i] = make_double2(0.0, 0.0);
}

__global__ void __launch_bounds__(256)
k_norm_partials_axial(const double2 *__restrict__ psi, int nr, long long count, double hr,
                      double *__restrict__ partials)
{
    __shared__ double red[32];
    double v = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const double2 u = psi[p];
        v += (((int)(p % nr)) + 0.5) * hr * fma(u.x, u.x, u.y * u.y);
    }
    const double r = block_sum(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// One warp per line k; fixed-order per-lane sums, a warp tree, one row per line.
__global__ void __launch_bounds__(256)
k_observables_axial(const double2 *__restrict__ psi, ObsArgs a, double hr,
                    double *__restrict__ rows)
{
    const int lane = threadIdx.x & 31;
    const long long line = (long long)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nr = a.nx, nz = a.ny;
    if (line >= nz) return;
    const int k = (int)line;
    const double2 *row = psi + line * nr;
    const bool has_z = k + 1 < nz;
    double s0 = 0, sr = 0, sv = 0, s4 = 0, kr = 0, kz = 0;
    for (int i = lane; i < nr; i += 32) {
        const double rho = (i + 0.5) * hr;
        const double2 v = row[i];
        const double am = fma(v.x, v.x, v.y * v.y);
        const double w = rho * am;
        s0 += w;
        sr = fma(a.x2[i], w, sr);
        sv = fma(a.vx[i], w, sv);
        s4 = fma(w, am, s4);
        const double2 nb = i + 1 < nr ? row[i + 1] : make_double2(0.0, 0.0);
        const double dx = nb.x - v.x, dy = nb.y - v.y;
        kr = fma(rho + 0.5 * hr, fma(dx, dx, dy * dy), kr);
        const double2 nz_ = has_z ? row[i + nr] : make_double2(0.0, 0.0);
        const double ex = nz_.x - v.x, ey = nz_.y - v.y;
        kz = fma(rho, fma(ex, ex, ey * ey), kz);
    }
    s0 = warp_sum(s0);
    sr = warp_sum(sr);
    sv = warp_sum(sv);
    s4 = warp_sum(s4);
    kr = warp_sum(kr);
    kz = warp_sum(kz);
    if (lane == 0) {
        const double sc = *a.scale, s2 = sc * sc;
        double *out = rows + line * kObsWidth;
        out[0] = s2 * s0;
        out[1] = s2 * sr;
        out[2] = 0.0;
        out[3] = s2 * a.y2[k] * s0;
        out[4] = s2 * (sv + a.vy[k] * s0);
        out[5] = s2 * s2 * s4;
        out[6] = s2 * kr;
        out[7] = s2 * kz;
        out[8] = 0.0;
    }
}

}  // namespace

void radial_tables(int m, double kre, double kim, double2 *cp_top, double2 *mult_top,
                   double2 *cp_bot, double2 *mult_bot, double *ka_top, double *kc_bot,
                   double2 *mid, double *ka_mid, double *kc_mid)
{
    using cd = std::complex<double>;
    const cd kappa(kre, kim);
    const double kabs = std::abs(kappa);
    auto a = [](int j) { return 1.0 - 1.0 / (2.0 * (j - 1) + 1.0); };   // unknown j = i + 1
    auto c = [](int j) { return 1.0 + 1.0 / (2.0 * (j - 1) + 1.0); };
    std::vector<cd> ct(m + 2, 0.0), cb(m + 2, 0.0);      // c'_j (top), e'_j (bottom), 1-based
    for (int j = 1; j <= m; ++j) {
        const cd f = 1.0 / (1.0 + 2.0 * kappa + kappa * a(j) * ct[j - 1]);
        ct[j] = -kappa * c(j) * f;
        mult_top[j - 1] = make_double2(f.real(), f.imag());
        cp_top[j - 1] = make_double2(ct[j].real(), ct[j].imag());
        ka_top[j - 1] = kabs * a(j);
    }
    for (int j = m; j >= 1; --j) {
        const cd f = 1.0 / (1.0 + 2.0 * kappa + kappa * c(j) * cb[j + 1]);
        cb[j] = -kappa * a(j) * f;
        mult_bot[m - j] = make_double2(f.real(), f.imag());
        cp_bot[m - j] = make_double2(cb[j].real(), cb[j].imag());
        kc_bot[m - j] = kabs * c(j);
    }
    const int k = (m + 1) / 2;
    const cd f = 1.0 / (1.0 + 2.0 * kappa + kappa * (a(k) * ct[k - 1] + c(k) * cb[k + 1]));
    *mid = make_double2(f.real(), f.imag());
    *ka_mid = kabs * a(k);
    *kc_mid = kabs * c(k);
}

int sweep_rho_blocks(int nz) { return (nz + kLinesPerBlock - 1) / kLinesPerBlock; }

cudaError_t launch_sweep_rho(int mode, void *psi, void *work, const RadialTables &rt, int nr,
                             int nz, const NonlinArgs &nl, cudaStream_t st)
{
    const int blocks = sweep_rho_blocks(nz);
    auto k = mode == 0 ? k_sweep_rho<0> : k_sweep_rho<1>;
    k<<<blocks, kThreads, 0, st>>>((double2 *)psi, (double2 *)work, rt, nr, nz, nl.px, nl.py,
                                   nl.pz, nl.g, nl.scale);
    return cudaGetLastError();
}

cudaError_t launch_seed_axial(void *psi, int nr, int nz, double hr, double hz, double gamma,
                              double lambda, cudaStream_t st)
{
    long long blocks = ((long long)nr * nz + 255) / 256;
    if (blocks > kReduceBlocks) blocks = kReduceBlocks;
    k_seed_axial<<<(int)blocks, 256, 0, st>>>((double2 *)psi, nr, nz, hr, hz, gamma, lambda);
    return cudaGetLastError();
}

cudaError_t launch_zero_axial(void *psi, int nr, cudaStream_t st)
{
    k_zero_axial<<<(nr + 255) / 256, 256, 0, st>>>((double2 *)psi, nr);
    return cudaGetLastError();
}

cudaError_t launch_norm_partials_axial(const void *psi, int nr, int nz, double hr,
                                       const Partials &out, int blocks, cudaStream_t st)
{
    k_norm_partials_axial<<<blocks, 256, 0, st>>>((const double2 *)psi, nr, (long long)nr * nz,
                                                  hr, out.buf);
    return cudaGetLastError();
}

cudaError_t launch_observables_axial(const void *psi, const ObsArgs &a, double hr,
                                     double *scratch, double *sums, cudaStream_t st)
{
    const long long lines = a.ny;
    double *rows = scratch, *stage = scratch + lines * kObsWidth;
    const long long blocks = (lines * 32 + 255) / 256;
    k_observables_axial<<<(unsigned)blocks, 256, 0, st>>>((const double2 *)psi, a, hr, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_rows_finish(rows, lines, stage, sums, st);
}

}  // namespace gp
