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

// calcnu of every point into pbuf (the radial windows overlap, so the
// pointwise step is taken once per point before them).  Blocks walk the
// radial lines (z index k), threads the points of a line: the line's factor
// P_z[k] and coefficients are set up once per line, not per point (FP64 work
// on GB300's narrow FP64 pipe, as was a 64-bit division per point).
template <int MODE>
__global__ void __launch_bounds__(256)
k_calcnu_axial(const double2 *__restrict__ in, double2 *__restrict__ pbuf, int nr, int nz,
               const double2 *__restrict__ pr, const double2 *__restrict__ pz,
               const double2 *__restrict__ one, StepG sg, const double *__restrict__ scale)
{
    const double G = sg.value();
    for (int k = blockIdx.x; k < nz; k += gridDim.x) {
        Calcnu<double, MODE> nl{};
        nl.setup(pr, pz, one, nullptr, nullptr, nullptr, k, 0, G, scale);
        const double2 *row = in + (long long)k * nr;
        double2 *out = pbuf + (long long)k * nr;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) out[i] = nl.apply(row[i], i);
    }
}

// Segmented-window radial sweep of pbuf (calcnu already applied): thread
// (q, k) owns core q of radial line k, solves rows a .. f (the core extended
// by W rows each side, clipped to the line) with the restarted tables of core
// q, and writes rows s .. e of out.
template <int MODE>
__global__ void __launch_bounds__(128)
k_sweep_rho_win(const double2 *__restrict__ pbuf, double2 *__restrict__ out,
                double2 *__restrict__ wscr, const SegWindow sw, int nr, int nz)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = (int)(tid % sw.nseg_r);
    const long long k = tid / sw.nseg_r;
    if (k >= nz) return;
    const int s = q * sw.Lc, e = min(nr, s + sw.Lc) - 1;
    const int a = max(0, s - sw.W), f = min(nr - 1, e + sw.W);
    const double2 *prow = pbuf + k * nr;
    double2 *rout = out + k * nr;
    double2 *w = wscr + (k * sw.nseg_r + q) * (long long)sw.W;
    const double2 *cpq = sw.cp_r + (long long)q * sw.tlen, *mq = sw.mult_r + (long long)q * sw.tlen;
    double2 d = make_double2(0.0, 0.0);
    for (int i0 = a; i0 <= f; i0 += kPrefetchR) {
        double2 pv[kPrefetchR];
#pragma unroll
        for (int u = 0; u < kPrefetchR; ++u)
            if (i0 + u <= f) pv[u] = prow[i0 + u];
#pragma unroll
        for (int u = 0; u < kPrefetchR; ++u) {
            const int i = i0 + u;
            if (i <= f) {
                d = LineOps<double, MODE>{sw.ka_r[i]}.fwd(pv[u], d, mq[i - a]);
                if (i >= s && i <= e) {
                    rout[i] = d;
                } else if (i > e) {
                    w[i - e - 1] = d;
                }
            }
        }
    }
    double2 v = d;
    for (int i = f; i >= s; --i) {
        if (i < f) v = LineOps<double, MODE>{0.0}.back(i > e ? w[i - e - 1] : rout[i], cpq[i - a], v);
        if (i <= e) rout[i] = LineOps<double, MODE>::out(v, prow[i]);
    }
}

// Segmented-window axial sweep along z: thread (i, q), rho index i fastest
// (neighbouring threads on neighbouring addresses), unknowns j = 1 .. nz - 1
// at stored row j.  Constant coefficients: the restarted tables of any core
// are the standard ones from its window's first row.
template <int MODE, bool NORM, bool NLOUT>
__global__ void __launch_bounds__(128)
k_sweep_z_win(const double2 *__restrict__ in, double2 *__restrict__ out,
              double2 *__restrict__ wscr, const SegWindow sw, const double2 *__restrict__ cp,
              const double2 *__restrict__ mult, double kap, int nr, int nz,
              const double2 *__restrict__ pz, const double2 *__restrict__ px,
              const double2 *__restrict__ p1, StepG sg, const double *__restrict__ rho_w,
              double *__restrict__ partials)
{
    __shared__ double red[32];
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(tid % nr);
    const long long q = tid / nr;
    const bool active = q < sw.nseg_z;
    const int m = nz - 1;
    double acc = 0.0;
    if (active) {
        const int s = 1 + (int)q * sw.Lc, e = min(m, s + sw.Lc - 1);
        const int a = max(1, s - sw.W), f = min(m, e + sw.W);
        double2 *w = wscr + ((long long)i * sw.nseg_z + q) * sw.W;
        const LineOps<double, MODE> cn{kap};
        Calcnu<double, MODE> nl{};
        if (NLOUT) nl.setup(pz, px, p1, nullptr, nullptr, nullptr, i, 0, sg.value(), nullptr);
        double2 d = make_double2(0.0, 0.0);
        for (int j0 = a; j0 <= f; j0 += kPrefetchR) {
            double2 pv[kPrefetchR];
#pragma unroll
            for (int u = 0; u < kPrefetchR; ++u)
                if (j0 + u <= f) pv[u] = in[(long long)(j0 + u) * nr + i];
#pragma unroll
            for (int u = 0; u < kPrefetchR; ++u) {
                const int j = j0 + u;
                if (j <= f) {
                    d = cn.fwd(pv[u], d, mult[j - a]);
                    if (j >= s && j <= e) out[(long long)j * nr + i] = d;
                    else if (j > e) w[j - e - 1] = d;
                }
            }
        }
        double2 v = d;
        for (int j = f; j >= s; --j) {
            if (j < f) v = cn.back(j > e ? w[j - e - 1] : out[(long long)j * nr + i], cp[j - a], v);
            if (j <= e) {
                double2 u = LineOps<double, MODE>::out(v, in[(long long)j * nr + i]);
                if (NLOUT) u = nl.apply(u, j);
                out[(long long)j * nr + i] = u;
                if (NORM) acc = fma(u.x, u.x, fma(u.y, u.y, acc));
            }
        }
        if (NORM) acc *= rho_w[i];
    }
    if (NORM) {
        const double r = block_sum(acc, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = r;
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

void radial_window_tables(int m, double kre, double kim, int Lc, int W, double2 *cp, double2 *mult,
                          double *ka)
{
    using cd = std::complex<double>;
    const cd kappa(kre, kim);
    const double kabs = std::abs(kappa);
    const int nseg = (m + Lc - 1) / Lc, tlen = Lc + 2 * W;
    auto a = [](int i) { return 1.0 - 1.0 / (2.0 * i + 1.0); };     // 0-based row i
    auto c = [](int i) { return 1.0 + 1.0 / (2.0 * i + 1.0); };
    for (int i = 0; i < m; ++i) ka[i] = kabs * a(i);
    for (int q = 0; q < nseg; ++q) {
        const int s = q * Lc, e = std::min(m, s + Lc) - 1;
        const int lo = std::max(0, s - W), hi = std::min(m - 1, e + W);
        cd prev = 0.0;
        for (int i = lo; i <= hi; ++i) {
            const cd f = 1.0 / (1.0 + 2.0 * kappa + kappa * a(i) * prev);
            prev = -kappa * c(i) * f;
            mult[(size_t)q * tlen + (i - lo)] = make_double2(f.real(), f.imag());
            cp[(size_t)q * tlen + (i - lo)] = make_double2(prev.real(), prev.imag());
        }
    }
}

int radial_window_width(int m, double kre, double kim, int Lc, double tol, int wmax)
{
    using cd = std::complex<double>;
    const cd kappa(kre, kim);
    std::vector<double> rb(m), rf(m);       // |c'_i|, |kappa a_i mult_i|
    cd prev = 0.0;
    for (int i = 0; i < m; ++i) {
        const double ai = 1.0 - 1.0 / (2.0 * i + 1.0), ci = 1.0 + 1.0 / (2.0 * i + 1.0);
        const cd f = 1.0 / (1.0 + 2.0 * kappa + kappa * ai * prev);
        prev = -kappa * ci * f;
        rb[i] = std::abs(prev);
        rf[i] = std::abs(kappa * ai * f);
    }
    for (int W = 1; W <= wmax; ++W) {
        bool ok = true;
        for (int s = 0; s < m && ok; s += Lc) {
            const int e = std::min(m, s + Lc) - 1;
            if (s - W > 0) {                  // forward truncation at row s - W
                double p = 1.0;
                for (int i = s - W; i < s; ++i) p *= rf[i];
                ok = p < tol;
            }
            if (ok && e + W < m - 1) {        // backward truncation after row e + W
                double p = 1.0;
                for (int i = e + 1; i <= e + W; ++i) p *= rb[i];
                ok = p < tol;
            }
        }
        if (ok) return W;
    }
    return 0;
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

cudaError_t launch_sweep_rho_win(int mode, const void *in, void *out, void *pbuf, void *wscr,
                                 const SegWindow &sw, int nr, int nz, const NonlinArgs &nl,
                                 cudaStream_t st)
{
    const int pb = nz < 16 * 152 ? nz : 16 * 152;    // one radial line per block at a time
    auto kc = mode == 0 ? k_calcnu_axial<0> : k_calcnu_axial<1>;
    kc<<<pb, 256, 0, st>>>((const double2 *)in, (double2 *)pbuf, nr, nz, nl.px, nl.py, nl.pz, nl.g,
                           nl.scale);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const long long threads = (long long)sw.nseg_r * nz;
    const int blocks = (int)((threads + 127) / 128);
    auto k = mode == 0 ? k_sweep_rho_win<0> : k_sweep_rho_win<1>;
    k<<<blocks, 128, 0, st>>>((const double2 *)pbuf, (double2 *)out, (double2 *)wscr, sw, nr, nz);
    return cudaGetLastError();
}

cudaError_t launch_sweep_z_win(int mode, const void *in, void *out, void *wscr,
                               const SegWindow &sw, const AxisTables &az, int nr, int nz,
                               const NonlinArgs *nlout, const double *rho_w,
                               const Partials *norm_out, int *blocks, cudaStream_t st)
{
    const long long threads = (long long)sw.nseg_z * nr;
    const int nb = (int)((threads + 127) / 128);
    if (blocks) *blocks = nb;
    const double kap = mode == 0 ? az.kre : az.kim;
    const StepG sg = nlout ? nlout->g : StepG{};
    const double2 *pz = nlout ? nlout->px : nullptr, *px = nlout ? nlout->py : nullptr,
                  *p1 = nlout ? nlout->pz : nullptr;
    double *part = norm_out ? norm_out->buf : nullptr;
#define GP_ZW(M, N, O)                                                                        \
    k_sweep_z_win<M, N, O><<<nb, 128, 0, st>>>((const double2 *)in, (double2 *)out,           \
                                               (double2 *)wscr, sw, az.cp64, az.mult64, kap,  \
                                               nr, nz, pz, px, p1, sg, rho_w, part)
    if (nlout) {
        if (mode != 1 || norm_out) return cudaErrorInvalidValue;
        GP_ZW(1, false, true);
    } else if (mode == 0) {
        if (norm_out) GP_ZW(0, true, false);
        else GP_ZW(0, false, false);
    } else {
        if (norm_out) GP_ZW(1, true, false);
        else GP_ZW(1, false, false);
    }
#undef GP_ZW
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
