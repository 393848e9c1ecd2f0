// gp_api.cu -- host side of libgp: the C ABI declared in include/gp.h, the
// per-context device state, the Crank-Nicolson coefficient tables and the
// CUDA-graph replay of the SSCN time loop.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gp.h"
#include "sscn_internal.h"
#include "sscn_slab.h"

using gp::AxisTables;
using gp::Partials;
using gp::SweepGeom;

struct gp_ctx {
    gp_grid grid{};
    double h[3]{}, dt = 0, w[3]{}, g = 0;
    int mode = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    void *psi = nullptr, *work = nullptr;
    AxisTables ax[2][3];            // [mode][axis]
    double2 *ph[2][3]{};            // [mode][axis] exp(-tau w_k^2 x^2 / 2)
    float4 *ph32[2][3]{};           // hi + lo pairs
    float *th32[3]{};               // dt w_k^2 x^2 / 2 per axis (FP32)
    double2 *phh[2][3]{};           // half-step factors exp(-tau w_k^2 x^2 / 4)
    float4 *phh32[2][3]{};
    float *thh32[3]{};              // dt w_k^2 x^2 / 4 (FP32)
    int split = GP_SPLIT_LIE;
    double g1 = 0, omega = 0;       // g(t) = g + g1 cos(omega t)
    long long *step_dev = nullptr;  // device step counter (modulated g)
    // axially symmetric psi(rho, z): grid {n_r, n_z, 1}, axis 0 = rho
    bool axial = false;
    gp::RadialTables rt[2];         // [mode] radial sweep tables (device)
    void *rt_mem[2]{};
    double *rho_w = nullptr;        // rho_i, the norm weights
    gp::SegWindow segw[2];          // [mode] segmented-window sweeps (few long lines)
    bool seg_ok[2]{};
    void *segw_mem[2]{};
    void *pbuf = nullptr, *wscr = nullptr;
    // FP64 real-time potential factor table (one psi-sized buffer, built on
    // the first real-time step that uses it)
    int pot_table = 1;
    double2 *pot3 = nullptr;        // exp(-i dt V) per point (plain splitting)
    double2 *pot3h = nullptr;       // exp(-i dt V / 2) per point (symmetric splitting)
    double *partials = nullptr;     // norm partials, >= max sweep blocks
    int partial_cap = 0;
    double *obs_partials = nullptr; // observables scratch (rows + finish stage)
    double *obs_tab = nullptr;      // x^2 and w^2 x^2 / 2 per axis
    float *obs_tab32 = nullptr;     // their FP32 roundings
    double *sums = nullptr;         // kObsWidth
    double *scale = nullptr;        // pending imaginary-time scale
    double *norm_dev = nullptr;     // last norm N
    int *err_dev = nullptr;         // device error bits
    double *host_sums = nullptr;    // pinned
    int *host_err = nullptr;        // pinned

    // float-float form (GP_CFF): expanded Crank-Nicolson and x-factor tables
    gp::FfAxis ffax[2][3];          // [mode][axis]
    gp::FfCoef *ffpx[2][3]{};       // [mode][axis] exp(-tau w_k^2 x^2 / 2), expanded
    void *ffmem = nullptr;          // one allocation for all of them
    float2 *obs_ff = nullptr;       // x_i^2, then w_x^2 x_i^2 / 2, as float-float pairs

    // z-slab of a grid split over several GPUs (gp_create_slab): local plane k
    // is global plane z0 + k of a z_global-plane grid
    bool slab = false;
    int slab_P = 1, slab_rank = 0, z_global = 0, z0 = 0, slab_nloc = 0;
    double2 *slab_consts = nullptr;    // device: the reduced system's two inverse rows (4 P)
    double2 *slab_spike = nullptr;     // device: s then t on the local unknown planes
    void *slab_saved = nullptr;        // device: psi on the first / last unknown plane
    double *slab_part = nullptr;       // device: interface reduction partials + result
    double *slab_host = nullptr;       // pinned: interface result

    CUtensorMap maps[3];            // 64-byte aligned type
    bool map_ok[3]{};
    bool tma_ok[2][3]{};            // [mode][axis] TMA path eligible
    int path_opt = GP_PATH_AUTO;
    int tile_shape = 0;

    int64_t step = 0;
    bool scale_pending = false;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    std::string last_error;
};

namespace {

thread_local std::string g_create_error;

constexpr int kGraphSteps = 10;

int fail(gp_ctx *c, int code, const std::string &msg)
{
    if (c) c->last_error = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(gp_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, m);
}

#define GP_CK(ctx, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

bool valid_grid(const gp_grid *g)
{
    if (!g) return false;
    auto ok = [](int n) { return n >= 3 && n <= GP_MAX_EDGE; };
    return ok(g->nx) && ok(g->ny) && (g->nz == 1 || ok(g->nz));
}

long long points(const gp_grid &g) { return (long long)g.nx * g.ny * g.nz; }

size_t elem_bytes(int prec) { return prec == GP_C64 ? 8 : 16; }

bool is_ff(const gp_ctx *c) { return c->prec == GP_CFF; }

// Number of float-float coefficients the context keeps: per mode and axis,
// c' and mult (m each) and the factor table (n).
size_t ff_coefs(const gp_grid &g)
{
    size_t n = 0;
    for (int k = 0; k < 3; ++k) {
        const size_t e = k == 0 ? g.nx : (k == 1 ? g.ny : g.nz);
        n += 2 * (2 * (e - 1 + (e == 1 ? 1 : 0)) + e);
    }
    return n;
}

double coord(int n, double h, int i) { return n == 1 ? 0.0 : -0.5 * n * h + i * h; }

int naxes(const gp_grid &g) { return g.nz > 1 ? 3 : 2; }

int edge(const gp_grid &g, int k) { return k == 0 ? g.nx : (k == 1 ? g.ny : g.nz); }

SweepGeom geom(const gp_grid &gr, int axis)
{
    const long long nx = gr.nx, ny = gr.ny;
    SweepGeom g{};
    if (axis == 0) { g.n = gr.nx; g.lines_a = gr.ny; g.lines_b = gr.nz; g.stride_a = nx; g.stride_b = nx * ny; g.pstride = 1; }
    else if (axis == 1) { g.n = gr.ny; g.lines_a = gr.nx; g.lines_b = gr.nz; g.stride_a = 1; g.stride_b = nx * ny; g.pstride = nx; }
    else { g.n = gr.nz; g.lines_a = gr.nx; g.lines_b = gr.ny; g.stride_a = 1; g.stride_b = nx; g.pstride = nx * ny; }
    return g;
}

double cell_volume(const gp_ctx *c)
{
    if (c->axial) return 2.0 * 3.14159265358979323846 * c->h[0] * c->h[1];
    return c->h[0] * c->h[1] * (c->grid.nz > 1 ? c->h[2] : 1.0);
}

// Coordinate of stored point i on axis k: the Cartesian grid, or on the axial
// grid's radial axis rho_i = (i + 1/2) h.
double axis_coord(const gp_ctx *c, int k, int i)
{
    if (c->axial && k == 0) return (i + 0.5) * c->h[0];
    if (c->slab && k == 2) return coord(c->z_global, c->h[2], c->z0 + i);
    return coord(edge(c->grid, k), c->h[k], i);
}

int alloc(gp_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    return GP_OK;
}

int upload_tables(gp_ctx *c)
{
    for (int mode = 0; mode < 2; ++mode) {
        for (int k = 0; k < naxes(c->grid); ++k) {
            AxisTables &a = c->ax[mode][k];
            const int n = edge(c->grid, k), m = n - 1;
            const double kap = c->dt / (4.0 * c->h[k] * c->h[k]);
            a.n = n;
            a.h = c->h[k];
            a.kre = mode == 0 ? kap : 0.0;
            a.kim = mode == 0 ? 0.0 : kap;
            std::vector<double2> cp(m), mult(m);
            std::vector<float4> cp32(m), mult32(m);
            double2 *d_cp64 = a.cp64, *d_mult64 = a.mult64;
            float4 *d_cp32 = a.cp32, *d_mult32 = a.mult32;
            gp::fill_tables(a, m, a.kre, a.kim, cp.data(), mult.data(), cp32.data(), mult32.data());
            GP_CK(c, cudaMemcpy(d_cp64, cp.data(), m * sizeof(double2), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(d_mult64, mult.data(), m * sizeof(double2), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(d_cp32, cp32.data(), m * sizeof(float4), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(d_mult32, mult32.data(), m * sizeof(float4), cudaMemcpyHostToDevice));
            if (is_ff(c)) {
                gp::FfAxis &f = c->ffax[mode][k];
                gp::FfCoef *d_cp = f.cp, *d_mult = f.mult;
                std::vector<gp::FfCoef> fcp(m), fmult(m);
                double cmax = 0.0;
                for (int i = 0; i < m; ++i) cmax = std::max(cmax, std::hypot(cp[i].x, cp[i].y));
                gp::ff_tables(m, cp.data(), mult.data(), a.conv64, cmax, kap, gp::ff_chunk(0), f,
                              fcp.data(), fmult.data());
                f.cp = d_cp;
                f.mult = d_mult;
                GP_CK(c, cudaMemcpy(d_cp, fcp.data(), m * sizeof(gp::FfCoef), cudaMemcpyHostToDevice));
                GP_CK(c, cudaMemcpy(d_mult, fmult.data(), m * sizeof(gp::FfCoef), cudaMemcpyHostToDevice));
            }
        }
    }
    {
        std::vector<double> x2, v;
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < edge(c->grid, k); ++i) {
                const double x = axis_coord(c, k, i);
                x2.push_back(x * x);
                v.push_back(0.5 * c->w[k] * c->w[k] * x * x);
            }
        x2.insert(x2.end(), v.begin(), v.end());
        GP_CK(c, cudaMemcpy(c->obs_tab, x2.data(), x2.size() * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<float> x2f(x2.begin(), x2.end());
        GP_CK(c, cudaMemcpy(c->obs_tab32, x2f.data(), x2f.size() * sizeof(float), cudaMemcpyHostToDevice));
        if (is_ff(c)) {
            const int nx = c->grid.nx, nt = c->grid.nx + c->grid.ny + c->grid.nz;
            std::vector<float2> t(2 * (size_t)nx);
            for (int i = 0; i < nx; ++i) {
                for (int q = 0; q < 2; ++q) {
                    const double v = x2[(size_t)q * nt + i];
                    const float h = (float)v;
                    t[(size_t)q * nx + i] = make_float2(h, (float)(v - (double)h));
                }
            }
            GP_CK(c, cudaMemcpy(c->obs_ff, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice));
        }
    }
    for (int mode = 0; mode < 2; ++mode) {
        for (int k = 0; k < 3; ++k) {
            const int n = edge(c->grid, k);
            std::vector<double2> t(n);
            std::vector<float4> t32(n);
            for (int i = 0; i < n; ++i) {
                const double x = axis_coord(c, k, i);
                const double th = c->dt * 0.5 * c->w[k] * c->w[k] * x * x;
                t[i] = mode == 0 ? make_double2(std::exp(-th), 0.0)
                                 : make_double2(std::cos(th), -std::sin(th));
                t32[i] = gp::split_coef(t[i]);
            }
            GP_CK(c, cudaMemcpy(c->ph[mode][k], t.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(c->ph32[mode][k], t32.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
            if (is_ff(c)) {
                std::vector<gp::FfCoef> tf(n);
                for (int i = 0; i < n; ++i) tf[i] = gp::ff_expand(t[i]);
                GP_CK(c, cudaMemcpy(c->ffpx[mode][k], tf.data(), n * sizeof(gp::FfCoef), cudaMemcpyHostToDevice));
            }
            for (int i = 0; i < n; ++i) {
                const double x = axis_coord(c, k, i);
                const double th = 0.5 * (c->dt * 0.5 * c->w[k] * c->w[k] * x * x);
                t[i] = mode == 0 ? make_double2(std::exp(-th), 0.0)
                                 : make_double2(std::cos(th), -std::sin(th));
                t32[i] = gp::split_coef(t[i]);
            }
            GP_CK(c, cudaMemcpy(c->phh[mode][k], t.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(c->phh32[mode][k], t32.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
        }
    }
    for (int k = 0; k < 3; ++k) {
        const int n = edge(c->grid, k);
        std::vector<float> th(n), thh(n);
        for (int i = 0; i < n; ++i) {
            const double x = axis_coord(c, k, i);
            th[i] = (float)(c->dt * 0.5 * c->w[k] * c->w[k] * x * x);
            thh[i] = 0.5f * th[i];
        }
        GP_CK(c, cudaMemcpy(c->th32[k], th.data(), n * sizeof(float), cudaMemcpyHostToDevice));
        GP_CK(c, cudaMemcpy(c->thh32[k], thh.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (c->axial) {
        const int m = c->grid.nx;
        const double kap = c->dt / (4.0 * c->h[0] * c->h[0]);
        for (int mode = 0; mode < 2; ++mode) {
            std::vector<double2> t4(4 * (size_t)m);
            std::vector<double> t2(2 * (size_t)m);
            gp::RadialTables &r = c->rt[mode];
            gp::radial_tables(m, mode == 0 ? kap : 0.0, mode == 0 ? 0.0 : kap, t4.data(),
                              t4.data() + m, t4.data() + 2 * m, t4.data() + 3 * m, t2.data(),
                              t2.data() + m, &r.mid, &r.ka_mid, &r.kc_mid);
            double2 *d4 = (double2 *)c->rt_mem[mode];
            double *d2 = (double *)(d4 + 4 * (size_t)m);
            GP_CK(c, cudaMemcpy(d4, t4.data(), t4.size() * sizeof(double2), cudaMemcpyHostToDevice));
            GP_CK(c, cudaMemcpy(d2, t2.data(), t2.size() * sizeof(double), cudaMemcpyHostToDevice));
            r.cp_top = d4;
            r.mult_top = d4 + m;
            r.cp_bot = d4 + 2 * m;
            r.mult_bot = d4 + 3 * m;
            r.ka_top = d2;
            r.kc_bot = d2 + m;
        }
        std::vector<double> rho(m);
        for (int i = 0; i < m; ++i) rho[i] = axis_coord(c, 0, i);
        GP_CK(c, cudaMemcpy(c->rho_w, rho.data(), m * sizeof(double), cudaMemcpyHostToDevice));
    }
    return GP_OK;
}

// Segmented-window sweeps of the axial form: one window W and core length Lc
// per mode, W the smallest that shields every core below 2^-55 from the
// truncated coupling on both axes; eligible when some axis gets >= 2 cores.
int setup_segments(gp_ctx *c)
{
    const int nr = c->grid.nx, nz = c->grid.ny, mz = nz - 1;
    size_t wscr_need = 0;
    for (int mode = 0; mode < 2; ++mode) {
        const double kap = c->dt / (4.0 * c->h[0] * c->h[0]);
        const double kre = mode == 0 ? kap : 0.0, kim = mode == 0 ? 0.0 : kap;
        const int wz = c->ax[mode][1].win64;
        int W = 0, Lc = 64;
        for (int it = 0; it < 4; ++it) {
            const int wr = gp::radial_window_width(nr, kre, kim, Lc, std::ldexp(1.0, -55), 256);
            W = (wr > 0 && wz > 0) ? std::max(wr, wz) : 0;
            if (W == 0 || Lc >= 2 * W) break;
            Lc = 2 * W;
        }
        gp::SegWindow &sw = c->segw[mode];
        sw = gp::SegWindow{};
        c->seg_ok[mode] = false;
        if (W == 0 || Lc < 2 * W) continue;
        sw.W = W;
        sw.Lc = Lc;
        sw.nseg_r = (nr + Lc - 1) / Lc;
        sw.nseg_z = (mz + Lc - 1) / Lc;
        sw.tlen = Lc + 2 * W;
        if (sw.nseg_r < 2 && sw.nseg_z < 2) continue;
        const size_t n2 = (size_t)sw.nseg_r * sw.tlen;
        std::vector<double2> cp(n2), mult(n2);
        std::vector<double> ka(nr);
        gp::radial_window_tables(nr, kre, kim, Lc, W, cp.data(), mult.data(), ka.data());
        int rc;
        if ((rc = alloc(c, &c->segw_mem[mode], 2 * n2 * sizeof(double2) + nr * sizeof(double)))) return rc;
        double2 *d2 = (double2 *)c->segw_mem[mode];
        double *dk = (double *)(d2 + 2 * n2);
        GP_CK(c, cudaMemcpy(d2, cp.data(), n2 * sizeof(double2), cudaMemcpyHostToDevice));
        GP_CK(c, cudaMemcpy(d2 + n2, mult.data(), n2 * sizeof(double2), cudaMemcpyHostToDevice));
        GP_CK(c, cudaMemcpy(dk, ka.data(), nr * sizeof(double), cudaMemcpyHostToDevice));
        sw.cp_r = d2;
        sw.mult_r = d2 + n2;
        sw.ka_r = dk;
        c->seg_ok[mode] = true;
        wscr_need = std::max(wscr_need, (size_t)W * std::max((size_t)nz * sw.nseg_r,
                                                              (size_t)nr * sw.nseg_z));
        // the axial sweep's norm partials: one per block
        const int zb = (int)(((long long)sw.nseg_z * nr + 127) / 128);
        if (zb > c->partial_cap) {
            double *bigger = nullptr;
            if ((rc = alloc(c, (void **)&bigger, (size_t)zb * sizeof(double)))) return rc;
            cudaFree(c->partials);
            c->partials = bigger;
            c->partial_cap = zb;
        }
    }
    if (c->seg_ok[0] || c->seg_ok[1]) {
        int rc;
        if ((rc = alloc(c, &c->pbuf, (size_t)nr * nz * sizeof(double2)))) return rc;
        if ((rc = alloc(c, &c->wscr, std::max<size_t>(wscr_need, 1) * sizeof(double2)))) return rc;
    }
    return GP_OK;
}

// TMA path eligibility per (mode, axis): the tensor map encodes, and the
// window truncation bound max|c'|^(C+1) is below the precision's rounding.
void setup_tma(gp_ctx *c)
{
    if (c->axial) {
        for (int k = 0; k < 3; ++k) {
            c->map_ok[k] = false;
            c->tma_ok[0][k] = c->tma_ok[1][k] = false;
        }
        return;
    }
    if (is_ff(c)) {
        for (int k = 0; k < naxes(c->grid); ++k) {
            c->map_ok[k] = gp::make_ff_map(c->tile_shape, c->psi, c->grid.nx, c->grid.ny,
                                           c->grid.nz, k, &c->maps[k]) == cudaSuccess;
            cudaGetLastError();
            for (int mode = 0; mode < 2; ++mode) {
                const int w = c->ffax[mode][k].win;
                c->tma_ok[mode][k] = c->map_ok[k] && w >= 1 && w <= gp::ff_chunk(c->tile_shape);
            }
        }
        return;
    }
    const int C = gp::tma_chunk(c->prec, c->tile_shape);
    for (int k = 0; k < naxes(c->grid); ++k) {
        c->map_ok[k] = gp::make_sweep_map(c->prec, c->tile_shape, c->psi, c->grid.nx, c->grid.ny,
                                          c->grid.nz, k, &c->maps[k]) == cudaSuccess;
        cudaGetLastError();
        for (int mode = 0; mode < 2; ++mode) {
            const gp::AxisTables &a = c->ax[mode][k];
            const int w = c->prec == GP_C64 ? a.win32 : a.win64;
            // complex64 runs one point behind the chunk: the seed must lie in
            // the part of chunk q already eliminated
            const int wmax = c->prec == GP_C64 ? C - 1 : C;
            c->tma_ok[mode][k] = c->map_ok[k] && w >= 1 && w <= wmax;
        }
    }
}

size_t footprint_bytes(const gp_grid &g, int prec)
{
    const size_t psi = (size_t)points(g) * elem_bytes(prec);
    size_t tables = 0;
    for (int k = 0; k < 3; ++k) {
        const size_t n = edge(g, k);
        tables += 2 * 2 * n * (sizeof(double2) + sizeof(float4)) + 2 * 2 * n * (sizeof(double2) + sizeof(float4)) +
                  2 * n * sizeof(float);
    }
    int blocks = 0;
    for (int k = 0; k < naxes(g); ++k) {
        for (int sh = 0; sh < gp::tma_shapes(prec); ++sh)
            blocks = std::max({blocks, gp::sweep_blocks(geom(g, k)), gp::tma_blocks(prec, sh, geom(g, k))});
        if (prec == GP_CFF)
            for (int sh = 0; sh < gp::ff_shapes(); ++sh) blocks = std::max(blocks, gp::ff_blocks(sh, geom(g, k)));
    }
    if (prec == GP_CFF) tables += ff_coefs(g) * sizeof(gp::FfCoef) + 2 * (size_t)g.nx * sizeof(float2);
    blocks = std::max(blocks, gp::kReduceBlocks);
    gp::ObsArgs oa{};
    oa.nx = g.nx;
    oa.ny = g.ny;
    oa.nz = g.nz;
    const size_t red = (size_t)blocks * sizeof(double) +
                       (size_t)gp::obs_scratch_doubles(oa) * sizeof(double) +
                       2 * (size_t)(g.nx + g.ny + g.nz) * sizeof(double) +
                       gp::kObsWidth * sizeof(double) + 2 * sizeof(double) + sizeof(int) +
                       sizeof(long long);
    // FP64: the real-time potential factor table (one more psi)
    return (prec == GP_C128 ? 3 : 2) * psi + tables + red;
}

// ---- float-float form: conversions at the boundary ------------------------

// psi <- scale * psi (float-float), scale <- 1, through the complex128 work buffer
cudaError_t ff_rescale(gp_ctx *c)
{
    const long long n = points(c->grid);
    cudaError_t e = gp::launch_ff_to_c128(c->work, c->psi, n, c->scale, c->stream);
    if (e == cudaSuccess) e = gp::launch_ff_from_c128(c->psi, c->work, n, nullptr, c->scale, c->stream);
    return e;
}

void release(gp_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(c->psi);
    fr(c->work);
    fr(c->ffmem);
    fr(c->slab_consts);
    fr(c->slab_spike);
    fr(c->slab_saved);
    fr(c->slab_part);
    if (c->slab_host) cudaFreeHost(c->slab_host);
    fr(c->obs_ff);
    for (auto &row : c->ax)
        for (auto &a : row) { fr(a.cp64); fr(a.mult64); fr(a.cp32); fr(a.mult32); }
    for (int mode = 0; mode < 2; ++mode)
        for (int k = 0; k < 3; ++k) {
            fr(c->ph[mode][k]);
            fr(c->ph32[mode][k]);
            fr(c->phh[mode][k]);
            fr(c->phh32[mode][k]);
        }
    for (int k = 0; k < 3; ++k) { fr(c->th32[k]); fr(c->thh32[k]); }
    fr(c->step_dev);
    fr(c->rt_mem[0]);
    fr(c->rt_mem[1]);
    fr(c->rho_w);
    fr(c->segw_mem[0]);
    fr(c->segw_mem[1]);
    fr(c->pbuf);
    fr(c->wscr);
    fr(c->pot3);
    fr(c->pot3h);
    fr(c->partials);
    fr(c->obs_partials);
    fr(c->obs_tab);
    fr(c->obs_tab32);
    fr(c->sums);
    fr(c->scale);
    fr(c->norm_dev);
    fr(c->err_dev);
    if (c->host_sums) cudaFreeHost(c->host_sums);
    if (c->host_err) cudaFreeHost(c->host_err);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Path of the sweep along `axis` in the current mode.
// x and y fused over z-planes in shared memory (3D Cartesian grids whose
// plane fits one CTA)
bool slab_ok(const gp_ctx *c)
{
    return !c->axial && !is_ff(c) && c->grid.nz > 1 && gp::slab_fits(c->prec, c->grid.nx, c->grid.ny);
}

int sweep_path(const gp_ctx *c, int axis)
{
    if (c->axial) {
        const bool seg = c->seg_ok[c->mode] && c->path_opt != GP_PATH_EXACT;
        return seg ? GP_PATH_WINDOW : GP_PATH_EXACT;
    }
    if (is_ff(c)) return GP_PATH_TMA;      // the float-float form has one sweep path
    if (c->path_opt == GP_PATH_SLAB && axis < 2 && slab_ok(c)) return GP_PATH_SLAB;
    if (!c->tma_ok[c->mode][axis]) return GP_PATH_EXACT;
    if (c->path_opt == GP_PATH_EXACT) return GP_PATH_EXACT;
    if (c->path_opt == GP_PATH_TMA) return GP_PATH_TMA;
    // auto: the FP64 path is bound by the FP64 pipe, where the window's extra
    // back-substitution work costs more than the traffic it saves
    return c->prec == GP_C64 ? GP_PATH_TMA : GP_PATH_EXACT;
}

cudaError_t launch_sweep(gp_ctx *c, int axis, const gp::NonlinArgs *nl, bool nl_at_output,
                         const Partials *norm, int *blocks)
{
    if (c->axial && axis == 0) {
        if (!nl || nl_at_output || norm) return cudaErrorInvalidValue;
        if (blocks) *blocks = gp::sweep_rho_blocks(c->grid.ny);
        return gp::launch_sweep_rho(c->mode, c->psi, c->work, c->rt[c->mode], c->grid.nx,
                                    c->grid.ny, *nl, c->stream);
    }
    const SweepGeom g = geom(c->grid, axis);
    const gp::AxisTables &ax = c->ax[c->mode][axis];
    if (is_ff(c)) {
        if (nl_at_output) return cudaErrorInvalidValue;
        gp::FfNonlin fn;
        if (nl) {
            fn.px = c->ffpx[c->mode][0];
            fn.py = nl->py;
            fn.pz = nl->pz;
            fn.g = nl->g;
            fn.scale = nl->scale;
        }
        if (blocks) *blocks = gp::ff_blocks(c->tile_shape, g);
        return gp::launch_sweep_ff(c->tile_shape, c->mode, axis, c->maps[axis], c->ffax[c->mode][axis],
                                   g, nl ? &fn : nullptr, norm, c->err_dev, c->stream);
    }
    if (sweep_path(c, axis) == GP_PATH_TMA) {
        if (blocks) *blocks = gp::tma_blocks(c->prec, c->tile_shape, g);
        return gp::launch_sweep_tma(c->prec, c->tile_shape, c->mode, axis, c->maps[axis], ax, g,
                                    nl, norm, c->err_dev, c->stream, nl_at_output);
    }
    if (blocks) *blocks = gp::sweep_blocks(g);
    if (nl && !nl_at_output)
        return gp::launch_sweep_x(c->prec, c->mode, c->psi, c->work, ax, g, *nl, c->grid.ny,
                                  c->grid.nz, norm, c->stream);
    return gp::launch_sweep_yz(c->prec, c->mode, c->psi, c->work, ax, g, norm, c->stream,
                               nl_at_output ? nl : nullptr);
}

bool modulated(const gp_ctx *c) { return c->g1 != 0.0; }

// calcnu of the part [fa dt, fb dt] of a step, for a sweep along `axis`: the
// factor tables along the axis first, then those of the line's (a, b) axes;
// half selects the half-step tables.
gp::NonlinArgs pointwise_args(const gp_ctx *c, int axis, bool half, double fa, double fb,
                              const double *scale)
{
    const int order[3] = {axis, axis == 0 ? 1 : 0, axis == 2 ? 1 : 2};
    const int mode = c->mode;
    gp::NonlinArgs nl;
    double2 *const *P = half ? c->phh[mode] : c->ph[mode];
    float4 *const *P32 = half ? c->phh32[mode] : c->ph32[mode];
    float *const *TH = half ? c->thh32 : c->th32;
    nl.px = P[order[0]];
    nl.py = P[order[1]];
    nl.pz = P[order[2]];
    nl.px32 = P32[order[0]];
    nl.py32 = P32[order[1]];
    nl.pz32 = P32[order[2]];
    nl.tx32 = TH[order[0]];
    nl.ty32 = TH[order[1]];
    nl.tz32 = TH[order[2]];
    nl.g.G = c->g * (fb - fa) * c->dt;
    if (modulated(c)) {
        nl.g.step = c->step_dev;
        nl.g.g0 = c->g;
        nl.g.g1 = c->g1;
        nl.g.omega = c->omega;
        nl.g.dt = c->dt;
        nl.g.fa = fa;
        nl.g.fb = fb;
    }
    nl.scale = scale;
    return nl;
}

// FP64 real-time steps on the exact path read their potential factors from a
// precomputed table: the full-step one for the plain splitting's x sweep, the
// half-step one for both half steps of the symmetric splitting.
bool uses_pot3(const gp_ctx *c)
{
    if (!c->pot_table || c->prec != GP_C128 || c->mode != GP_REAL || c->axial) return false;
    for (int k = 0; k < naxes(c->grid); ++k)
        if (sweep_path(c, k) != GP_PATH_EXACT) return false;
    return true;
}

double2 *pot3_for(const gp_ctx *c) { return c->split == GP_SPLIT_STRANG ? c->pot3h : c->pot3; }

// Allocate and fill the table this step needs (never under stream capture).
int prepare_pot3(gp_ctx *c)
{
    if (!uses_pot3(c) || pot3_for(c)) return GP_OK;
    const bool half = c->split == GP_SPLIT_STRANG;
    double2 **slot = half ? &c->pot3h : &c->pot3;
    int rc = alloc(c, (void **)slot, (size_t)points(c->grid) * sizeof(double2));
    if (rc) return rc;
    double2 *const *P = half ? c->phh[GP_REAL] : c->ph[GP_REAL];
    GP_CK(c, gp::launch_build_pot3(*slot, P[0], P[1], P[2], c->grid.nx, c->grid.ny, c->grid.nz,
                                   c->stream));
    return GP_OK;
}

// Enqueue one SSCN step.  With ev != nullptr, record ev[0] before the first
// kernel and ev[1 + k] after kernel slot k (x, y, z sweep, then the norm
// finish and the rest of the step); slots a step does not launch get their
// event recorded back to back.
//   plain (Lie): calcnu(dt) fused into the x sweep; y, z sweeps; imaginary
//                time: norm partials in the last sweep, norm finish.
//   symmetric:   calcnu(dt/2) in the x sweep; y, z sweeps; calcnu(dt/2) fused
//                into the last sweep's stores (real time), or (imaginary time)
//                norm finish, calcnu(dt/2) pass with norm partials, norm finish.
int enqueue_step(gp_ctx *c, cudaEvent_t *ev = nullptr)
{
    const int mode = c->mode;
    const bool three_d = c->grid.nz > 1;
    const bool strang = c->split == GP_SPLIT_STRANG;
    const bool imag = mode == GP_IMAG;
    const int last = three_d ? 2 : 1;
    Partials part{c->partials, 1, c->axial ? c->rho_w : nullptr};
    gp::NonlinArgs nl = pointwise_args(c, 0, strang, 0.0, strang ? 0.5 : 1.0, c->scale);
    gp::NonlinArgs nl2 =
        pointwise_args(c, imag ? 0 : last, true, 0.5, 1.0, imag ? c->scale : nullptr);
    if (uses_pot3(c) && pot3_for(c)) {
        nl.p3 = pot3_for(c);
        if (!imag) nl2.p3 = pot3_for(c);
    }
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], c->stream) : cudaSuccess; };
    GP_CK(c, mark(0));
    int last_blocks = 0;
    if (c->axial && sweep_path(c, 0) == GP_PATH_WINDOW) {
        // psi -> work (radial), work -> psi (axial): neighbouring cores read
        // each other's rows, so each sweep writes another buffer
        const gp::SegWindow &sw = c->segw[mode];
        GP_CK(c, gp::launch_sweep_rho_win(mode, c->psi, c->work, c->pbuf, c->wscr, sw, c->grid.nx,
                                          c->grid.ny, nl, c->stream));
        GP_CK(c, mark(1));
        const bool out_nl = strang && !imag;
        GP_CK(c, gp::launch_sweep_z_win(mode, c->work, c->psi, c->wscr, sw, c->ax[mode][1],
                                        c->grid.nx, c->grid.ny, out_nl ? &nl2 : nullptr, c->rho_w,
                                        imag ? &part : nullptr, &last_blocks, c->stream));
        GP_CK(c, mark(2));
        GP_CK(c, mark(3));
    } else {
    const bool slab = sweep_path(c, 0) == GP_PATH_SLAB;
    if (slab) {
        GP_CK(c, gp::launch_sweep_xy(c->prec, mode, c->psi, c->grid.nx, c->grid.ny, c->grid.nz,
                                     c->ax[mode][0], c->ax[mode][1], nl, c->stream));
        GP_CK(c, mark(1));
        GP_CK(c, mark(2));
    } else {
        GP_CK(c, launch_sweep(c, 0, &nl, false, nullptr, nullptr));
        GP_CK(c, mark(1));
    }
    for (int axis = slab ? 2 : 1; axis <= last; ++axis) {
        const bool is_last = axis == last;
        const gp::NonlinArgs *out_nl = (is_last && strang && !imag) ? &nl2 : nullptr;
        GP_CK(c, launch_sweep(c, axis, out_nl, out_nl != nullptr,
                              (is_last && imag) ? &part : nullptr, &last_blocks));
        GP_CK(c, mark(axis + 1));
    }
    if (!three_d) GP_CK(c, mark(3));
    }
    if (imag) {
        GP_CK(c, gp::launch_norm_finish(c->partials, last_blocks, cell_volume(c), c->scale,
                                        c->norm_dev, c->err_dev, c->stream));
        if (strang) {
            GP_CK(c, gp::launch_calcnu_pass(c->prec, mode, c->psi, c->grid.nx, c->grid.ny,
                                            c->grid.nz, nl2, part, gp::kReduceBlocks, c->stream,
                                            c->axial ? c->rho_w : nullptr));
            GP_CK(c, gp::launch_norm_finish(c->partials, gp::kReduceBlocks, cell_volume(c),
                                            c->scale, c->norm_dev, c->err_dev, c->stream));
        }
    }
    if (modulated(c)) GP_CK(c, gp::launch_add_step(c->step_dev, c->stream));
    GP_CK(c, mark(4));
    return GP_OK;
}

// Kernel launches per step (for launch accounting).
int kernels_per_step(const gp_ctx *c)
{
    const bool imag = c->mode == GP_IMAG, strang = c->split == GP_SPLIT_STRANG;
    const bool seg = c->axial && sweep_path(c, 0) == GP_PATH_WINDOW;   // + the calcnu pass
    const bool slab = sweep_path(c, 0) == GP_PATH_SLAB;      // x and y in one launch
    return (c->grid.nz > 1 ? 3 : 2) - (slab ? 1 : 0) + (seg ? 1 : 0) + (imag ? 1 : 0) +
           (imag && strang ? 2 : 0) + (modulated(c) ? 1 : 0);
}

void drop_graph(gp_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_steps = 0;
}

// Capture kGraphSteps steps into a graph; on any capture failure fall back
// to plain launches (graph stays null).
void build_graph(gp_ctx *c)
{
    drop_graph(c);
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int rc = GP_OK;
    for (int s = 0; s < kGraphSteps && rc == GP_OK; ++s) rc = enqueue_step(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != GP_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
        c->graph = ex;
        c->graph_steps = kGraphSteps;
    } else {
        cudaGetLastError();
    }
    cudaGraphDestroy(g);
}

int materialize_scale(gp_ctx *c)
{
    if (!c->scale_pending) return GP_OK;
    if (is_ff(c)) GP_CK(c, ff_rescale(c));
    else GP_CK(c, gp::launch_apply_scale(c->prec, c->psi, points(c->grid), c->scale, c->stream));
    c->scale_pending = false;
    return GP_OK;
}

gp::ObsArgs obs_args(const gp_ctx *c)
{
    gp::ObsArgs a{};
    a.nx = c->grid.nx;
    a.ny = c->grid.ny;
    a.nz = c->grid.nz;
    a.x2 = c->obs_tab;
    a.y2 = a.x2 + c->grid.nx;
    a.z2 = a.y2 + c->grid.ny;
    a.vx = a.z2 + c->grid.nz;
    a.vy = a.vx + c->grid.nx;
    a.vz = a.vy + c->grid.ny;
    a.x2f = c->obs_tab32;
    a.vxf = c->obs_tab32 + (c->grid.nx + c->grid.ny + c->grid.nz);
    a.scale = c->scale;
    return a;
}

// Observables pass and finish, then the 9 sums to pinned host memory.
int enqueue_observables(gp_ctx *c)
{
    if (c->axial)
        GP_CK(c, gp::launch_observables_axial(c->psi, obs_args(c), c->h[0], c->obs_partials,
                                              c->sums, c->stream));
    else if (is_ff(c))
        GP_CK(c, gp::launch_observables_ff(c->psi, obs_args(c), c->obs_ff, c->obs_ff + c->grid.nx,
                                           c->obs_partials, c->sums, c->stream));
    else
        GP_CK(c, gp::launch_observables(c->prec, c->psi, obs_args(c), c->obs_partials, c->sums,
                                        c->stream));
    GP_CK(c, cudaMemcpyAsync(c->host_sums, c->sums, gp::kObsWidth * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    return GP_OK;
}

int read_errors(gp_ctx *c)
{
    GP_CK(c, cudaMemcpyAsync(c->host_err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP_CK(c, cudaStreamSynchronize(c->stream));
    if (*c->host_err & 2) return fail(c, GP_ETIMEOUT, "a sweep's bounded wait for a TMA chunk gave up");
    if (*c->host_err & 1) return fail(c, GP_ENONFINITE, "norm became non-finite or zero");
    return GP_OK;
}

}  // namespace

void gp::set_thread_error(const char *msg) { g_create_error = msg ? msg : ""; }

void gp::host_thomas_tables(int m, double kre, double kim, double2 *cp, double2 *mult)
{
    double2 prev = make_double2(0.0, 0.0);
    for (int i = 0; i < m; ++i) {
        thomas_step(kre, kim, prev.x, prev.y, mult[i], cp[i]);
        prev = cp[i];
    }
}

float4 gp::split_coef(double2 v)
{
    const float hx = (float)v.x, hy = (float)v.y;
    return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

namespace {

// Middle-row multiplier of the two-ended elimination,
// 1 / (1 + 2 kappa + kappa (c'_{k-1} + c'_{m-k})), k = ceil(m / 2), c'_0 = 0.
double2 mid_multiplier(int m, std::complex<double> kappa, const double2 *cp)
{
    const int k = (m + 1) / 2;
    auto c = [&](int j) {
        return j <= 0 ? std::complex<double>(0.0) : std::complex<double>(cp[j - 1].x, cp[j - 1].y);
    };
    const std::complex<double> f = 1.0 / (1.0 + 2.0 * kappa + kappa * (c(k - 1) + c(m - k)));
    return make_double2(f.real(), f.imag());
}

// Smallest W with cmax^(W+1) < tol (0 if none up to 64).
int window_for(double cmax, double tol)
{
    double p = cmax;
    for (int w = 1; w <= 64; ++w) {
        p *= cmax;
        if (p < tol) return w;
    }
    return 0;
}

}  // namespace

void gp::fill_tables(AxisTables &a, int m, double kre, double kim, double2 *cp64, double2 *mult64,
                     float4 *cp32, float4 *mult32)
{
    a.kre = kre;
    a.kim = kim;
    host_thomas_tables(m, kre, kim, cp64, mult64);
    const double kre32 = (double)(float)kre, kim32 = (double)(float)kim;
    std::vector<double2> cpf(m), mf(m);
    host_thomas_tables(m, kre32, kim32, cpf.data(), mf.data());
    for (int i = 0; i < m; ++i) {
        cp32[i] = split_coef(cpf[i]);
        mult32[i] = split_coef(mf[i]);
    }
    a.mid64 = mid_multiplier(m, std::complex<double>(kre, kim), cp64);
    a.mid32 = split_coef(mid_multiplier(m, std::complex<double>(kre32, kim32), cpf.data()));
    // convergence: from conv on, every entry equals the last one
    auto eq64 = [](double2 p, double2 q) { return p.x == q.x && p.y == q.y; };
    auto eq32 = [](float4 p, float4 q) { return p.x == q.x && p.y == q.y && p.z == q.z && p.w == q.w; };
    int c64 = m - 1, c32 = m - 1;
    while (c64 > 0 && eq64(cp64[c64 - 1], cp64[m - 1]) && eq64(mult64[c64 - 1], mult64[m - 1])) --c64;
    while (c32 > 0 && eq32(cp32[c32 - 1], cp32[m - 1]) && eq32(mult32[c32 - 1], mult32[m - 1])) --c32;
    a.conv64 = c64;
    a.conv32 = c32;
    a.cinf64 = cp64[m - 1];
    a.minf64 = mult64[m - 1];
    a.cinf32 = cp32[m - 1];
    a.minf32 = mult32[m - 1];
    double cmax64 = 0.0, cmax32 = 0.0;
    for (int i = 0; i < m; ++i) {
        cmax64 = std::max(cmax64, std::hypot(cp64[i].x, cp64[i].y));
        cmax32 = std::max(cmax32, std::hypot(cpf[i].x, cpf[i].y));
    }
    // The window's truncation is the same linear perturbation at every step,
    // so it is held far below one rounding: over 10^4 sweeps it stays under
    // ~1e-8 (complex64) and ~1e-12 (FP64) of the norm in real time.
    a.win64 = window_for(cmax64, std::ldexp(1.0, -55));
    a.win32 = window_for(cmax32, std::ldexp(1.0, -40));
}

// =================================================================== C ABI

extern "C" {

int gp_footprint(const gp_grid *grid, int precision, size_t *bytes)
{
    if (!valid_grid(grid) || (precision != GP_C128 && precision != GP_C64 && precision != GP_CFF) ||
        !bytes)
        return fail(nullptr, GP_EINVAL, "gp_footprint: invalid grid or precision");
    *bytes = footprint_bytes(*grid, precision);
    return GP_OK;
}

namespace {
// Where a z-slab context sits in its grid (gp_create_slab).
struct SlabSpec {
    int P, rank, z_global, z0;
};
int create_ctx(const gp_grid *grid, const double dx[3], double dt, double gamma, double nu,
               double lambda, double g, int mode, int precision, void *cuda_stream, bool axial,
               gp_ctx **out, const SlabSpec *slab = nullptr);
}

int gp_create(const gp_grid *grid, const double dx[3], double dt, double gamma, double nu,
              double lambda, double g, int mode, int precision, void *cuda_stream,
              gp_ctx **out)
{
    if (out) *out = nullptr;
    if (!out || !valid_grid(grid) || !dx)
        return fail(nullptr, GP_EINVAL, "gp_create: invalid grid (nx, ny >= 3; nz == 1 or >= 3; <= 8192)");
    const int nd = grid->nz > 1 ? 3 : 2;
    for (int k = 0; k < nd; ++k)
        if (!(dx[k] > 0) || !std::isfinite(dx[k])) return fail(nullptr, GP_EINVAL, "gp_create: dx must be > 0");
    return create_ctx(grid, dx, dt, gamma, nu, lambda, g, mode, precision, cuda_stream, false, out);
}

int gp_create_axial(int nr, int nz, double hr, double hz, double dt, double gamma, double lambda,
                    double g, int mode, int precision, void *cuda_stream, gp_ctx **out)
{
    if (out) *out = nullptr;
    const gp_grid grid{nr, nz, 1};
    if (!out || !valid_grid(&grid))
        return fail(nullptr, GP_EINVAL, "gp_create_axial: need 3 <= n_r, n_z <= 8192");
    if (!(hr > 0) || !(hz > 0) || !std::isfinite(hr + hz))
        return fail(nullptr, GP_EINVAL, "gp_create_axial: h_r, h_z must be > 0");
    if (precision != GP_C128)
        return fail(nullptr, GP_EINVAL, "gp_create_axial: the axially symmetric form is FP64 (GP_C128)");
    const double dx[3] = {hr, hz, 1.0};
    return create_ctx(&grid, dx, dt, gamma, lambda, 0.0, g, mode, precision, cuda_stream, true, out);
}

int gp_footprint_axial(int nr, int nz, int precision, size_t *bytes)
{
    const gp_grid grid{nr, nz, 1};
    if (!valid_grid(&grid) || precision != GP_C128 || !bytes)
        return fail(nullptr, GP_EINVAL, "gp_footprint_axial: invalid grid or precision");
    // + radial tables, rho weights, and (segmented windows) the core buffer,
    // the window scratch (W <= Lc / 2 rows per core: at most one psi), the
    // restarted tables and the axial sweep's norm partials
    const size_t psi = (size_t)nr * nz * sizeof(double2);
    *bytes = footprint_bytes(grid, precision) + 2 * (size_t)nr * (4 * sizeof(double2) + 2 * sizeof(double)) +
             (size_t)nr * sizeof(double) + 2 * psi +
             2 * (2 * (size_t)(2 * nr + 512) * sizeof(double2) + (size_t)nr * sizeof(double)) +
             ((size_t)(nz / 32 + 2) * nr / 128 + 1) * sizeof(double);
    return GP_OK;
}

namespace {
int create_ctx(const gp_grid *grid, const double dx[3], double dt, double gamma, double nu,
               double lambda, double g, int mode, int precision, void *cuda_stream, bool axial,
               gp_ctx **out, const SlabSpec *slab)
{
    const int nd = grid->nz > 1 ? 3 : 2;
    if (!(dt > 0) || !std::isfinite(dt)) return fail(nullptr, GP_EINVAL, "gp_create: dt must be > 0");
    if (!(gamma >= 0) || !(nu >= 0) || !(lambda >= 0) || !std::isfinite(gamma + nu + lambda) ||
        !std::isfinite(g))
        return fail(nullptr, GP_EINVAL, "gp_create: trap frequencies must be >= 0 and g finite");
    if (mode != GP_IMAG && mode != GP_REAL) return fail(nullptr, GP_EINVAL, "gp_create: bad mode");
    if (precision != GP_C128 && precision != GP_C64 && (precision != GP_CFF || axial))
        return fail(nullptr, GP_EINVAL, "gp_create: bad precision");

    gp_ctx *c = new (std::nothrow) gp_ctx;
    if (!c) return fail(nullptr, GP_ENOMEM, "gp_create: host allocation failed");
    c->grid = *grid;
    c->h[0] = dx[0];
    c->h[1] = dx[1];
    c->h[2] = nd == 3 ? dx[2] : 1.0;
    c->dt = dt;
    c->w[0] = gamma;
    c->w[1] = nu;
    c->w[2] = nd == 3 ? lambda : 0.0;
    c->g = g;
    c->mode = mode;
    c->prec = precision;
    c->axial = axial;
    if (slab) {
        c->slab = true;
        c->slab_P = slab->P;
        c->slab_rank = slab->rank;
        c->z_global = slab->z_global;
        c->z0 = slab->z0;
    }

    auto bail = [&](int rc) {
        g_create_error = c->last_error;
        release(c);
        delete c;
        return rc;
    };
    int rc;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
        c->own_stream = true;
    }
    const size_t psi_bytes = (size_t)points(c->grid) * elem_bytes(precision);
    if ((rc = alloc(c, &c->psi, psi_bytes))) return bail(rc);
    if ((rc = alloc(c, &c->work, psi_bytes))) return bail(rc);
    for (int mode_i = 0; mode_i < 2; ++mode_i)
        for (int k = 0; k < naxes(c->grid); ++k) {
            AxisTables &a = c->ax[mode_i][k];
            const size_t m = edge(c->grid, k) - 1;
            if ((rc = alloc(c, (void **)&a.cp64, m * sizeof(double2)))) return bail(rc);
            if ((rc = alloc(c, (void **)&a.mult64, m * sizeof(double2)))) return bail(rc);
            if ((rc = alloc(c, (void **)&a.cp32, m * sizeof(float4)))) return bail(rc);
            if ((rc = alloc(c, (void **)&a.mult32, m * sizeof(float4)))) return bail(rc);
        }
    for (int mode_i = 0; mode_i < 2; ++mode_i)
        for (int k = 0; k < 3; ++k) {
            const size_t n = edge(c->grid, k);
            if ((rc = alloc(c, (void **)&c->ph[mode_i][k], n * sizeof(double2)))) return bail(rc);
            if ((rc = alloc(c, (void **)&c->ph32[mode_i][k], n * sizeof(float4)))) return bail(rc);
            if ((rc = alloc(c, (void **)&c->phh[mode_i][k], n * sizeof(double2)))) return bail(rc);
            if ((rc = alloc(c, (void **)&c->phh32[mode_i][k], n * sizeof(float4)))) return bail(rc);
        }
    for (int k = 0; k < 3; ++k) {
        if ((rc = alloc(c, (void **)&c->th32[k], edge(c->grid, k) * sizeof(float)))) return bail(rc);
        if ((rc = alloc(c, (void **)&c->thh32[k], edge(c->grid, k) * sizeof(float)))) return bail(rc);
    }
    if (precision == GP_CFF) {
        if ((rc = alloc(c, &c->ffmem, ff_coefs(c->grid) * sizeof(gp::FfCoef)))) return bail(rc);
        if ((rc = alloc(c, (void **)&c->obs_ff, 2 * (size_t)c->grid.nx * sizeof(float2)))) return bail(rc);
        gp::FfCoef *q = static_cast<gp::FfCoef *>(c->ffmem);
        for (int mode_i = 0; mode_i < 2; ++mode_i)
            for (int k = 0; k < 3; ++k) {
                const int n = edge(c->grid, k);
                if (k < naxes(c->grid)) {
                    c->ffax[mode_i][k].cp = q;
                    q += n - 1;
                    c->ffax[mode_i][k].mult = q;
                    q += n - 1;
                }
                c->ffpx[mode_i][k] = q;
                q += n;
            }
    }
    if ((rc = alloc(c, (void **)&c->step_dev, sizeof(long long)))) return bail(rc);
    if (axial) {
        const size_t m = grid->nx;
        for (int mode_i = 0; mode_i < 2; ++mode_i)
            if ((rc = alloc(c, &c->rt_mem[mode_i], m * (4 * sizeof(double2) + 2 * sizeof(double)))))
                return bail(rc);
        if ((rc = alloc(c, (void **)&c->rho_w, m * sizeof(double)))) return bail(rc);
    }
    int blocks = gp::kReduceBlocks;
    for (int k = 0; k < naxes(c->grid); ++k) {
        for (int sh = 0; sh < gp::tma_shapes(precision); ++sh)
            blocks = std::max({blocks, gp::sweep_blocks(geom(c->grid, k)),
                               gp::tma_blocks(precision, sh, geom(c->grid, k))});
        if (precision == GP_CFF)
            for (int sh = 0; sh < gp::ff_shapes(); ++sh)
                blocks = std::max(blocks, gp::ff_blocks(sh, geom(c->grid, k)));
    }
    c->partial_cap = blocks;
    if ((rc = alloc(c, (void **)&c->partials, blocks * sizeof(double)))) return bail(rc);
    {
        gp::ObsArgs oa{};
        oa.nx = grid->nx;
        oa.ny = grid->ny;
        oa.nz = grid->nz;
        if ((rc = alloc(c, (void **)&c->obs_partials, gp::obs_scratch_doubles(oa) * sizeof(double)))) return bail(rc);
        const int nt = grid->nx + grid->ny + grid->nz;
        if ((rc = alloc(c, (void **)&c->obs_tab, 2 * nt * sizeof(double)))) return bail(rc);
        if ((rc = alloc(c, (void **)&c->obs_tab32, 2 * nt * sizeof(float)))) return bail(rc);
    }
    if ((rc = alloc(c, (void **)&c->sums, gp::kObsWidth * sizeof(double)))) return bail(rc);
    if ((rc = alloc(c, (void **)&c->scale, sizeof(double)))) return bail(rc);
    if ((rc = alloc(c, (void **)&c->norm_dev, sizeof(double)))) return bail(rc);
    if ((rc = alloc(c, (void **)&c->err_dev, sizeof(int)))) return bail(rc);
    {
        cudaError_t e = cudaMallocHost((void **)&c->host_sums, gp::kObsWidth * sizeof(double));
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
        e = cudaMallocHost((void **)&c->host_err, sizeof(int));
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
    }
    if ((rc = upload_tables(c))) return bail(rc);
    if (axial && (rc = setup_segments(c))) return bail(rc);
    setup_tma(c);
    if (precision == GP_CFF)
        for (int mode_i = 0; mode_i < 2; ++mode_i)
            for (int k = 0; k < naxes(c->grid); ++k)
                if (!c->tma_ok[mode_i][k]) {
                    fail(c, GP_EINVAL, "gp_create: the float-float form needs every axis's "
                                       "back-substitution window within one chunk "
                                       "(max|c'|^9 < 2^-50, about dt / (4 h^2) < 0.02)");
                    return bail(GP_EINVAL);
                }
    {
        cudaError_t e = cudaMemsetAsync(c->psi, 0, psi_bytes, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->step_dev, 0, sizeof(long long), c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
        const double one = 1.0;
        e = cudaMemcpyAsync(c->scale, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "init"));
    }
    *out = c;
    return GP_OK;
}
}  // namespace

int gp_load(gp_ctx *c, const void *psi, int64_t count, int on_device)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_load: null context");
    if (c->slab && !psi) return fail(c, GP_EINVAL, "gp_load: a z-slab seeds with gp_slab_seed");
    const long long n = points(c->grid);
    c->scale_pending = false;
    c->step = 0;
    GP_CK(c, gp::launch_set_step(c->step_dev, 0, c->stream));
    if (psi == nullptr) {
        Partials part{c->partials, 1};
        if (c->axial) {
            GP_CK(c, gp::launch_seed_axial(c->psi, c->grid.nx, c->grid.ny, c->h[0], c->h[1],
                                           c->w[0], c->w[1], c->stream));
            GP_CK(c, gp::launch_norm_partials_axial(c->psi, c->grid.nx, c->grid.ny, c->h[0], part,
                                                    gp::kReduceBlocks, c->stream));
        } else if (is_ff(c)) {
            // the seed in FP64 in the work buffer, normalised into psi
            GP_CK(c, gp::launch_seed(GP_C128, c->work, c->grid.nx, c->grid.ny, c->grid.nz, c->h,
                                     c->w, c->stream));
            GP_CK(c, gp::launch_norm_partials(GP_C128, c->work, n, part, gp::kReduceBlocks,
                                              c->stream));
            GP_CK(c, gp::launch_norm_finish(c->partials, gp::kReduceBlocks, cell_volume(c), c->scale,
                                            c->norm_dev, c->err_dev, c->stream));
            GP_CK(c, gp::launch_ff_from_c128(c->psi, c->work, n, c->scale, c->scale, c->stream));
            return GP_OK;
        } else {
            GP_CK(c, gp::launch_seed(c->prec, c->psi, c->grid.nx, c->grid.ny, c->grid.nz, c->h,
                                     c->w, c->stream));
            GP_CK(c, gp::launch_norm_partials(c->prec, c->psi, n, part, gp::kReduceBlocks,
                                              c->stream));
        }
        GP_CK(c, gp::launch_norm_finish(c->partials, gp::kReduceBlocks, cell_volume(c), c->scale,
                                        c->norm_dev, c->err_dev, c->stream));
        c->scale_pending = true;
        return materialize_scale(c);
    }
    if (count != n) return fail(c, GP_EINVAL, "gp_load: count != nx*ny*nz");
    if (is_ff(c)) {
        // complex128 in, split into float-float pairs with the Dirichlet
        // nodes zeroed (a device buffer is read in place, a host one first
        // crosses into the work buffer)
        const void *src = psi;
        if (!on_device) {
            GP_CK(c, cudaMemcpyAsync(c->work, psi, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice,
                                     c->stream));
            src = c->work;
        }
        GP_CK(c, gp::launch_ff_from_c128_grid(c->psi, src, c->grid.nx, c->grid.ny, c->grid.nz, c->stream));
        const double one = 1.0;
        GP_CK(c, cudaMemcpyAsync(c->scale, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        GP_CK(c, cudaStreamSynchronize(c->stream));   // `one` and the caller's buffer
        return GP_OK;
    }
    GP_CK(c, cudaMemcpyAsync(c->psi, psi, (size_t)n * elem_bytes(c->prec),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
    if (c->axial) GP_CK(c, gp::launch_zero_axial(c->psi, c->grid.nx, c->stream));
    else GP_CK(c, gp::launch_zero_boundary(c->prec, c->psi, c->grid.nx, c->grid.ny, c->grid.nz, c->stream));
    const double one = 1.0;
    GP_CK(c, cudaMemcpyAsync(c->scale, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    GP_CK(c, cudaStreamSynchronize(c->stream));   // `one` and the caller's buffer
    return GP_OK;
}

int gp_store(gp_ctx *c, void *out, int64_t count, int on_device)
{
    if (!c || !out) return fail(c, GP_EINVAL, "gp_store: null argument");
    const long long n = points(c->grid);
    if (count != n) return fail(c, GP_EINVAL, "gp_store: count != nx*ny*nz");
    if (is_ff(c)) {
        // hi + lo in FP64, times the pending scale
        void *dst = on_device ? out : c->work;
        GP_CK(c, gp::launch_ff_to_c128(dst, c->psi, n, c->scale, c->stream));
        if (!on_device)
            GP_CK(c, cudaMemcpyAsync(out, c->work, (size_t)n * sizeof(double2), cudaMemcpyDeviceToHost,
                                     c->stream));
        return read_errors(c);
    }
    int rc = materialize_scale(c);
    if (rc) return rc;
    GP_CK(c, cudaMemcpyAsync(out, c->psi, (size_t)n * elem_bytes(c->prec),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    return read_errors(c);
}

int gp_set_params(gp_ctx *c, double g, int mode)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_set_params: null context");
    if (!std::isfinite(g) || (mode != GP_IMAG && mode != GP_REAL))
        return fail(c, GP_EINVAL, "gp_set_params: bad g or mode");
    if (c->slab && mode != GP_REAL)
        return fail(c, GP_EINVAL, "gp_set_params: a z-slab runs in real time");
    if (mode != c->mode) {
        int rc = materialize_scale(c);
        if (rc) return rc;
    }
    c->g = g;
    c->mode = mode;
    drop_graph(c);
    return GP_OK;
}

int gp_set_modulation(gp_ctx *c, double g1, double omega)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_set_modulation: null context");
    if (!std::isfinite(g1) || !std::isfinite(omega))
        return fail(c, GP_EINVAL, "gp_set_modulation: g1 and omega must be finite");
    c->g1 = g1;
    c->omega = omega;
    GP_CK(c, gp::launch_set_step(c->step_dev, c->step, c->stream));
    drop_graph(c);
    return GP_OK;
}

int gp_step(gp_ctx *c, int64_t n)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_step: null context");
    if (c->slab) return fail(c, GP_EINVAL, "gp_step: a z-slab steps with gp_slab_step_begin / _end");
    if (n < 0) return fail(c, GP_EINVAL, "gp_step: n < 0");
    if (n == 0) return GP_OK;
    if (int rc = prepare_pot3(c)) return rc;
    if (n >= kGraphSteps && !c->graph) build_graph(c);
    int64_t done = 0;
    if (c->graph) {
        for (; done + c->graph_steps <= n; done += c->graph_steps)
            GP_CK(c, cudaGraphLaunch(c->graph, c->stream));
    }
    for (; done < n; ++done) {
        int rc = enqueue_step(c);
        if (rc) return rc;
    }
    c->step += n;
    if (c->mode == GP_IMAG) c->scale_pending = true;
    return GP_OK;
}

namespace {
// N, mu, E and the rms sizes from the 9 sums of the observables pass
// (complex64: K_k; otherwise R_k in place of K_k).
void finish_observables(const gp_ctx *c, const double *sums, gp_obs *o)
{
    double s[gp::kObsWidth];
    std::memcpy(s, sums, sizeof(s));
    if (c->prec != GP_C64 && !c->axial)
        for (int k = 6; k < 9; ++k) s[k] = 2.0 * s[0] - 2.0 * s[k];     // K_k from R_k
    const double w = cell_volume(c);
    const double n = w * s[0];
    double kin = 0.5 * (s[6] / (c->h[0] * c->h[0]) + s[7] / (c->h[1] * c->h[1]));
    if (c->grid.nz > 1) kin += 0.5 * s[8] / (c->h[2] * c->h[2]);
    // g at the current time (modulated: g + g1 cos(omega t))
    const double g_now = modulated(c) ? c->g + c->g1 * std::cos(c->omega * (c->step * c->dt)) : c->g;
    o->norm = n;
    o->mu = w * (kin + s[4] + g_now * s[5]) / n;
    o->energy = w * (kin + s[4] + 0.5 * g_now * s[5]) / n;
    if (c->axial) {
        // s[1] = sum rho^2 (weighted), s[3] = sum z^2: <x^2> = <y^2> = <rho^2> / 2
        o->rms_x = std::sqrt(0.5 * s[1] / s[0]);
        o->rms_y = o->rms_x;
        o->rms_z = std::sqrt(s[3] / s[0]);
        o->rms_r = std::sqrt((s[1] + s[3]) / s[0]);
    } else {
        o->rms_x = std::sqrt(s[1] / s[0]);
        o->rms_y = std::sqrt(s[2] / s[0]);
        o->rms_z = std::sqrt(s[3] / s[0]);
        o->rms_r = std::sqrt((s[1] + s[2] + s[3]) / s[0]);
    }
    o->step = c->step;
    o->t = c->step * c->dt;
}
}  // namespace

int gp_observables(gp_ctx *c, gp_obs *o)
{
    if (!c || !o) return fail(c, GP_EINVAL, "gp_observables: null argument");
    if (c->slab) return fail(c, GP_EINVAL, "gp_observables: a z-slab needs the sums of every rank (gp_slab_*)");
    int rc0 = enqueue_observables(c);
    if (rc0) return rc0;
    int rc = read_errors(c);
    finish_observables(c, c->host_sums, o);
    if (rc) return rc;
    const double v[7] = {o->norm, o->mu, o->energy, o->rms_x, o->rms_y, o->rms_z, o->rms_r};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, GP_ENONFINITE, "gp_observables: non-finite result");
    return GP_OK;
}

int gp_time_kernels(gp_ctx *c, int64_t steps, double *ms_out, int n_out)
{
    if (!c || !ms_out || n_out < 5 || steps < 1 || c->slab)
        return fail(c, GP_EINVAL, "gp_time_kernels: need steps >= 1 and n_out >= 5 (not on a z-slab)");
    if (int rc0 = prepare_pot3(c)) return rc0;
    cudaEvent_t ev[5];
    for (auto &e : ev) GP_CK(c, cudaEventCreate(&e));
    double acc[4] = {0, 0, 0, 0};
    int rc = GP_OK;
    for (int64_t s = 0; s < steps && rc == GP_OK; ++s) {
        rc = enqueue_step(c, ev);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(ev[4]);
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "cudaEventSynchronize"); break; }
        for (int k = 0; k < 4; ++k) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            acc[k] += ms;
        }
    }
    if (rc == GP_OK) {
        c->step += steps;
        if (c->mode == GP_IMAG) c->scale_pending = true;
        // one observables pass: the kernel, then its fixed-order finish
        cudaEvent_t e0 = ev[0], e1 = ev[1];
        cudaEventRecord(e0, c->stream);
        rc = enqueue_observables(c);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        for (int k = 0; k < 4; ++k) ms_out[k] = acc[k] / (double)steps;
        ms_out[4] = ms;
        for (int k = 5; k < n_out; ++k) ms_out[k] = 0.0;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

int gp_set_option(gp_ctx *c, int option, int value)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_set_option: null context");
    if (option == GP_OPT_SPLITTING) {
        if (value != GP_SPLIT_LIE && value != GP_SPLIT_STRANG)
            return fail(c, GP_EINVAL, "gp_set_option: unknown splitting");
        if (value == GP_SPLIT_STRANG && is_ff(c))
            return fail(c, GP_EINVAL, "gp_set_option: the float-float form runs the plain splitting");
        if (value == GP_SPLIT_STRANG && c->slab)
            return fail(c, GP_EINVAL, "gp_set_option: a z-slab runs the plain splitting");
        c->split = value;
        drop_graph(c);
        return GP_OK;
    }
    if (option == GP_OPT_POTENTIAL_TABLE) {
        if (value != 0 && value != 1) return fail(c, GP_EINVAL, "gp_set_option: potential table is 0 or 1");
        c->pot_table = value;
        if (!value && (c->pot3 || c->pot3h)) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->pot3);
            cudaFree(c->pot3h);
            c->pot3 = c->pot3h = nullptr;
        }
        drop_graph(c);
        return GP_OK;
    }
    if (option == GP_OPT_TILE_SHAPE) {
        if (value < 0 || value >= (is_ff(c) ? gp::ff_shapes() : gp::tma_shapes(c->prec)))
            return fail(c, GP_EINVAL, "gp_set_option: tile shape out of range");
        const int old = c->tile_shape;
        c->tile_shape = value;
        setup_tma(c);
        if (is_ff(c) && !c->tma_ok[c->mode][0]) {
            c->tile_shape = old;
            setup_tma(c);
            return fail(c, GP_EINVAL, "gp_set_option: tile shape does not apply to this grid");
        }
        if (c->path_opt == GP_PATH_TMA)
            for (int k = 0; k < naxes(c->grid); ++k)
                if (!c->tma_ok[c->mode][k]) c->path_opt = GP_PATH_AUTO;
        drop_graph(c);
        return GP_OK;
    }
    if (option != GP_OPT_SWEEP_PATH) return fail(c, GP_EINVAL, "gp_set_option: unknown option");
    if (value != GP_PATH_AUTO && value != GP_PATH_EXACT && value != GP_PATH_TMA &&
        value != GP_PATH_WINDOW && value != GP_PATH_SLAB)
        return fail(c, GP_EINVAL, "gp_set_option: unknown sweep path");
    if (value == GP_PATH_SLAB && !slab_ok(c))
        return fail(c, GP_EINVAL, "gp_set_option: the slab path needs a 3D Cartesian grid whose "
                                  "xy-plane fits one CTA's shared memory");
    if (value == GP_PATH_WINDOW && (!c->axial || !c->seg_ok[c->mode]))
        return fail(c, GP_EINVAL, "gp_set_option: the segmented-window path is for axial grids "
                                  "with long enough lines");
    if (value == GP_PATH_TMA && c->axial)
        return fail(c, GP_EINVAL, "gp_set_option: no TMA sweep path on the axial form");
    if (is_ff(c) && value != GP_PATH_AUTO && value != GP_PATH_TMA)
        return fail(c, GP_EINVAL, "gp_set_option: the float-float form has the TMA sweep path only");
    if (value == GP_PATH_TMA)
        for (int k = 0; k < naxes(c->grid); ++k)
            if (!c->tma_ok[c->mode][k])
                return fail(c, GP_EINVAL, "gp_set_option: the TMA sweep path does not apply to "
                                          "this grid, dt and mode");
    c->path_opt = value;
    drop_graph(c);
    return GP_OK;
}

int gp_autotune(gp_ctx *c, int steps, int *path_out, int *shape_out, double *ms_out)
{
    if (!c || steps < 1 || c->slab) return fail(c, GP_EINVAL, "gp_autotune: need steps >= 1 (not on a z-slab)");
    const size_t bytes = (size_t)points(c->grid) * elem_bytes(c->prec);
    void *saved = nullptr;
    double *saved_scale = nullptr;
    GP_CK(c, cudaMalloc(&saved, bytes));
    cudaError_t e = cudaMalloc((void **)&saved_scale, sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(saved);
        return cuda_fail(c, e, "cudaMalloc");
    }
    auto cleanup = [&]() {
        cudaFree(saved);
        cudaFree(saved_scale);
    };
    const int path0 = c->path_opt, shape0 = c->tile_shape;
    const int64_t step0 = c->step;
    const bool pending0 = c->scale_pending;
    e = cudaMemcpyAsync(saved, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved_scale, c->scale, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(c, e, "gp_autotune: save state");
    }
    struct Cand { int path, shape; };
    std::vector<Cand> cands;
    if (!is_ff(c)) cands.push_back({GP_PATH_EXACT, shape0});
    if (c->axial && c->seg_ok[c->mode]) cands.push_back({GP_PATH_WINDOW, shape0});
    if (slab_ok(c)) cands.push_back({GP_PATH_SLAB, shape0});
    for (int sh = 0; sh < (is_ff(c) ? gp::ff_shapes() : gp::tma_shapes(c->prec)); ++sh) {
        c->tile_shape = sh;
        setup_tma(c);
        bool ok = true;
        for (int k = 0; k < naxes(c->grid); ++k) ok = ok && c->tma_ok[c->mode][k];
        if (ok) cands.push_back({GP_PATH_TMA, sh});
    }
    if (cands.empty()) {
        cleanup();
        return fail(c, GP_EINTERNAL, "gp_autotune: no eligible sweep path");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    Cand pick = cands[0];
    int rc = GP_OK;
    for (const Cand &cd : cands) {
        c->tile_shape = cd.shape;
        setup_tma(c);
        c->path_opt = cd.path;
        drop_graph(c);
        if ((rc = prepare_pot3(c))) break;
        if ((rc = enqueue_step(c))) break;             // warm-up
        cudaEventRecord(e0, c->stream);
        for (int s = 0; s < steps && rc == GP_OK; ++s) rc = enqueue_step(c);
        cudaEventRecord(e1, c->stream);
        if (rc) break;
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = cd;
        }
        // back to the saved state for the next candidate
        cudaMemcpyAsync(c->psi, saved, bytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(c->scale, saved_scale, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (gp::launch_set_step(c->step_dev, step0, c->stream) != cudaSuccess && rc == GP_OK)
        rc = fail(c, GP_ECUDA, "gp_autotune: restore the step counter");
    e = cudaStreamSynchronize(c->stream);
    cleanup();
    c->step = step0;
    c->scale_pending = pending0;
    if (rc == GP_OK && e != cudaSuccess) rc = cuda_fail(c, e, "gp_autotune");
    if (rc != GP_OK) {
        c->path_opt = path0;
        c->tile_shape = shape0;
        setup_tma(c);
        drop_graph(c);
        return rc;
    }
    c->tile_shape = pick.shape;
    setup_tma(c);
    c->path_opt = pick.path;
    drop_graph(c);
    if (path_out) *path_out = pick.path;
    if (shape_out) *shape_out = pick.shape;
    if (ms_out) *ms_out = best / steps;
    return GP_OK;
}

int gp_get_option(gp_ctx *c, int option, int *value)
{
    if (!c || !value) return fail(c, GP_EINVAL, "gp_get_option: null argument");
    if (option == GP_OPT_SWEEP_PATH) *value = c->path_opt;
    else if (option == GP_OPT_TILE_SHAPE) *value = c->tile_shape;
    else if (option == GP_OPT_SPLITTING) *value = c->split;
    else if (option == GP_OPT_POTENTIAL_TABLE) *value = c->pot_table;
    else return fail(c, GP_EINVAL, "gp_get_option: unknown option");
    return GP_OK;
}

int gp_tile_shapes(int precision, int *count)
{
    if ((precision != GP_C128 && precision != GP_C64 && precision != GP_CFF) || !count)
        return fail(nullptr, GP_EINVAL, "gp_tile_shapes: bad precision");
    *count = precision == GP_CFF ? gp::ff_shapes() : gp::tma_shapes(precision);
    return GP_OK;
}

int gp_sweep_paths(gp_ctx *c, int path[3])
{
    if (!c || !path) return fail(c, GP_EINVAL, "gp_sweep_paths: null argument");
    for (int k = 0; k < 3; ++k) path[k] = k < naxes(c->grid) ? sweep_path(c, k) : 0;
    return GP_OK;
}

int gp_launches_per_step(gp_ctx *c, int *per_step, int *per_observables)
{
    if (!c) return fail(c, GP_EINVAL, "gp_launches_per_step: null context");
    if (per_step) *per_step = kernels_per_step(c);
    if (per_observables) *per_observables = 3;   // line pass + two finish passes
    return GP_OK;
}

int gp_sync(gp_ctx *c)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_sync: null context");
    return read_errors(c);
}

int gp_apply_pending_scale(gp_ctx *c)
{
    if (!c) return fail(nullptr, GP_EINVAL, "gp_apply_pending_scale: null context");
    return materialize_scale(c);
}

int gp_device_psi(gp_ctx *c, void **p)
{
    if (!c || !p) return fail(c, GP_EINVAL, "gp_device_psi: null argument");
    *p = c->psi;
    return GP_OK;
}

const char *gp_last_error(const gp_ctx *c)
{
    return c ? c->last_error.c_str() : g_create_error.c_str();
}

void gp_destroy(gp_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}


// ------------------------------------------------------------------ z-slabs

namespace {
// Solve (I - kappa L) x = b (m unknowns) with the host FP64 tables (the same
// recurrence as the device tables).
void host_solve(int m, const double2 *cp, const double2 *mult, std::complex<double> kappa,
                const std::vector<std::complex<double>> &b, std::vector<std::complex<double>> &x)
{
    std::vector<std::complex<double>> d(m);
    std::complex<double> prev = 0.0;
    for (int i = 0; i < m; ++i) {
        prev = (b[i] + kappa * prev) * std::complex<double>(mult[i].x, mult[i].y);
        d[i] = prev;
    }
    x.assign(m, 0.0);
    x[m - 1] = d[m - 1];
    for (int i = m - 2; i >= 0; --i) x[i] = d[i] - std::complex<double>(cp[i].x, cp[i].y) * x[i + 1];
}

// s = A^{-1} (kappa e_first), t = A^{-1} (kappa e_last) of an m-unknown block
void spikes(int m, double kim, std::vector<std::complex<double>> &s, std::vector<std::complex<double>> &t)
{
    std::vector<double2> cp(m), mult(m);
    gp::host_thomas_tables(m, 0.0, kim, cp.data(), mult.data());
    const std::complex<double> kappa(0.0, kim);
    std::vector<std::complex<double>> b(m, 0.0);
    b[0] = kappa;
    host_solve(m, cp.data(), mult.data(), kappa, b, s);
    b[0] = 0.0;
    b[m - 1] = kappa;
    host_solve(m, cp.data(), mult.data(), kappa, b, t);
}

long long slab_plane(const gp_ctx *c) { return (long long)c->grid.nx * c->grid.ny; }

// The reduced system of the boundary values, the same on every z line: with
// unknowns L_q (q = 0 .. P-2) at index 2q and F_q (q = 1 .. P-1) at 2q - 1,
//     L_q - sL_q L_{q-1} - tL_q F_{q+1} = yL_q,   F_q - sF_q L_{q-1} - tF_q F_{q+1} = yF_q.
// w <- the rows of its inverse that give L_{rank-1} (w[0 .. 2P)) and
// F_{rank+1} (w[2P .. 4P)), each as weights of the gathered values in their
// layout (rank q's yF at 2q, yL at 2q + 1); false if the matrix is singular.
bool reduced_rows(int P, int rank, const std::vector<std::complex<double>> &sF,
                  const std::vector<std::complex<double>> &sL, const std::vector<std::complex<double>> &tF,
                  const std::vector<std::complex<double>> &tL, std::vector<double2> &w)
{
    using cd = std::complex<double>;
    const int n = 2 * (P - 1);
    auto iL = [](int q) { return 2 * q; };
    auto iF = [](int q) { return 2 * q - 1; };
    std::vector<cd> a((size_t)n * n, 0.0), inv((size_t)n * n, 0.0);
    auto A = [&](int r, int k) -> cd & { return a[(size_t)r * n + k]; };
    auto X = [&](int r, int k) -> cd & { return inv[(size_t)r * n + k]; };
    for (int q = 0; q < P; ++q) {
        if (q <= P - 2) {
            A(iL(q), iL(q)) = 1.0;
            if (q >= 1) A(iL(q), iL(q - 1)) = -sL[q];
            A(iL(q), iF(q + 1)) = -tL[q];
        }
        if (q >= 1) {
            A(iF(q), iF(q)) = 1.0;
            A(iF(q), iL(q - 1)) = -sF[q];
            if (q <= P - 2) A(iF(q), iF(q + 1)) = -tF[q];
        }
    }
    for (int r = 0; r < n; ++r) X(r, r) = 1.0;
    // Gauss-Jordan with partial pivoting
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::abs(A(r, col)) > std::abs(A(piv, col))) piv = r;
        if (std::abs(A(piv, col)) == 0.0) return false;
        for (int k = 0; k < n; ++k) {
            std::swap(A(col, k), A(piv, k));
            std::swap(X(col, k), X(piv, k));
        }
        const cd d = A(col, col);
        for (int k = 0; k < n; ++k) {
            A(col, k) /= d;
            X(col, k) /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const cd f = A(r, col);
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A(r, k) -= f * A(col, k);
                X(r, k) -= f * X(col, k);
            }
        }
    }
    // column of the unknown's equation -> slot of its right-hand side
    auto slot = [&](int k) { return (k % 2 == 0) ? 2 * (k / 2) + 1 : 2 * ((k + 1) / 2); };
    const int rows[2] = {rank >= 1 ? iL(rank - 1) : -1, rank <= P - 2 ? iF(rank + 1) : -1};
    for (int h = 0; h < 2; ++h) {
        if (rows[h] < 0) continue;
        for (int k = 0; k < n; ++k) {
            const cd v = X(rows[h], k);
            w[(size_t)h * 2 * P + slot(k)] = make_double2(v.real(), v.imag());
        }
    }
    return true;
}
}  // namespace

int gp_create_slab(const gp_grid *global, const double dx[3], double dt, double gamma, double nu,
                   double lambda, double g, int nranks, const int *bounds, int rank,
                   void *cuda_stream, gp_ctx **out)
{
    if (out) *out = nullptr;
    if (!out || !valid_grid(global) || global->nz < 3 || !dx || !bounds)
        return fail(nullptr, GP_EINVAL, "gp_create_slab: invalid grid (3D) or null argument");
    if (nranks < 1 || nranks > gp::kSlabMaxRanks || rank < 0 || rank >= nranks)
        return fail(nullptr, GP_EINVAL, "gp_create_slab: 1 <= nranks <= 8 and 0 <= rank < nranks");
    if (bounds[0] != 0 || bounds[nranks] != global->nz)
        return fail(nullptr, GP_EINVAL, "gp_create_slab: bounds must run from 0 to nz");
    for (int q = 0; q < nranks; ++q) {
        const int unknowns = bounds[q + 1] - bounds[q] - (q == 0 ? 1 : 0);
        if (unknowns < 2) return fail(nullptr, GP_EINVAL, "gp_create_slab: every slab needs >= 2 unknown planes");
    }
    for (int k = 0; k < 3; ++k)
        if (!(dx[k] > 0) || !std::isfinite(dx[k])) return fail(nullptr, GP_EINVAL, "gp_create_slab: dx must be > 0");
    const int nzl = rank == 0 ? bounds[1] : bounds[rank + 1] - bounds[rank] + 1;
    const gp_grid local{global->nx, global->ny, nzl};
    const SlabSpec spec{nranks, rank, global->nz, rank == 0 ? 0 : bounds[rank] - 1};
    gp_ctx *c = nullptr;
    int rc = create_ctx(&local, dx, dt, gamma, nu, lambda, g, GP_REAL, GP_C128, cuda_stream, false, &c, &spec);
    if (rc) return rc;
    // spikes of every rank's block: the reduced matrix, this rank's spikes
    const double kim = dt / (4.0 * dx[2] * dx[2]);
    std::vector<std::complex<double>> sF(nranks), sL(nranks), tF(nranks), tL(nranks), s, t;
    for (int q = 0; q < nranks && !rc; ++q) {
        const int m = bounds[q + 1] - bounds[q] - (q == 0 ? 1 : 0);
        spikes(m, kim, s, t);
        sF[q] = s[0];
        sL[q] = s[m - 1];
        tF[q] = t[0];
        tL[q] = t[m - 1];
        if (q == rank) {
            c->slab_nloc = m;
            std::vector<double2> sp(2 * (size_t)m);
            for (int i = 0; i < m; ++i) {
                sp[i] = make_double2(s[i].real(), s[i].imag());
                sp[m + i] = make_double2(t[i].real(), t[i].imag());
            }
            if ((rc = alloc(c, (void **)&c->slab_spike, sp.size() * sizeof(double2)))) break;
            cudaError_t e = cudaMemcpy(c->slab_spike, sp.data(), sp.size() * sizeof(double2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = cuda_fail(c, e, "gp_create_slab: spikes");
        }
    }
    std::vector<double2> w(4 * (size_t)nranks, make_double2(0.0, 0.0));
    if (!rc && nranks > 1 && !reduced_rows(nranks, rank, sF, sL, tF, tL, w))
        rc = fail(c, GP_EINVAL, "gp_create_slab: singular reduced system");
    const long long plane = slab_plane(c);
    if (!rc) rc = alloc(c, (void **)&c->slab_consts, w.size() * sizeof(double2));
    if (!rc) {
        cudaError_t e = cudaMemcpy(c->slab_consts, w.data(), w.size() * sizeof(double2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "gp_create_slab: reduced rows");
    }
    if (!rc) rc = alloc(c, &c->slab_saved, 2 * (size_t)plane * sizeof(double2));
    if (!rc) rc = alloc(c, (void **)&c->slab_part, (gp::kReduceBlocks + 1) * sizeof(double));
    if (!rc) {
        cudaError_t e = cudaMallocHost((void **)&c->slab_host, sizeof(double));
        if (e != cudaSuccess) rc = cuda_fail(c, e, "cudaMallocHost");
    }
    if (rc) {
        g_create_error = c->last_error;
        gp_destroy(c);
        return rc;
    }
    *out = c;
    return GP_OK;
}

int gp_slab_exchange_count(gp_ctx *c, int64_t *count)
{
    if (!c || !c->slab || !count) return fail(c, GP_EINVAL, "gp_slab_exchange_count: not a z-slab");
    *count = 2 * slab_plane(c);
    return GP_OK;
}

int gp_slab_seed(gp_ctx *c)
{
    if (!c || !c->slab) return fail(c, GP_EINVAL, "gp_slab_seed: not a z-slab");
    c->step = 0;
    c->scale_pending = false;
    GP_CK(c, gp::launch_set_step(c->step_dev, 0, c->stream));
    GP_CK(c, gp::launch_slab_seed(c->psi, c->grid.nx, c->grid.ny, c->grid.nz, c->z_global, c->z0, c->h,
                                  c->w, c->stream));
    return GP_OK;
}

int gp_slab_scale(gp_ctx *c, double factor)
{
    if (!c || !c->slab || !std::isfinite(factor)) return fail(c, GP_EINVAL, "gp_slab_scale: bad argument");
    GP_CK(c, cudaMemcpyAsync(c->scale, &factor, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    GP_CK(c, gp::launch_apply_scale(GP_C128, c->psi, points(c->grid), c->scale, c->stream));
    GP_CK(c, cudaStreamSynchronize(c->stream));   // `factor`
    return GP_OK;
}

int gp_slab_step_begin(gp_ctx *c, void *bnd)
{
    if (!c || !c->slab || !bnd) return fail(c, GP_EINVAL, "gp_slab_step_begin: not a z-slab or null buffer");
    if (int rc = prepare_pot3(c)) return rc;
    const long long plane = slab_plane(c);
    const int kl = c->grid.nz - 1;
    gp::NonlinArgs nl = pointwise_args(c, 0, false, 0.0, 1.0, c->scale);
    if (uses_pot3(c) && pot3_for(c)) nl.p3 = pot3_for(c);
    GP_CK(c, launch_sweep(c, 0, &nl, false, nullptr, nullptr));
    GP_CK(c, launch_sweep(c, 1, nullptr, false, nullptr, nullptr));
    GP_CK(c, gp::launch_slab_capture(c->psi, c->slab_saved, plane, 1, kl, c->stream));
    GP_CK(c, launch_sweep(c, 2, nullptr, false, nullptr, nullptr));
    GP_CK(c, gp::launch_slab_bnd(c->psi, c->slab_saved, bnd, plane, 1, kl, c->stream));
    return GP_OK;
}

int gp_slab_step_end(gp_ctx *c, const void *bnd_all)
{
    if (!c || !c->slab || !bnd_all) return fail(c, GP_EINVAL, "gp_slab_step_end: not a z-slab or null buffer");
    GP_CK(c, gp::launch_slab_correct(c->psi, bnd_all, c->slab_consts, c->slab_spike, c->slab_P,
                                     slab_plane(c), c->slab_nloc, c->stream));
    if (modulated(c)) GP_CK(c, gp::launch_add_step(c->step_dev, c->stream));
    c->step += 1;
    return GP_OK;
}

int gp_slab_first_plane(gp_ctx *c, void *out)
{
    if (!c || !c->slab || !out) return fail(c, GP_EINVAL, "gp_slab_first_plane: not a z-slab or null buffer");
    const long long plane = slab_plane(c);
    GP_CK(c, cudaMemcpyAsync(out, static_cast<double2 *>(c->psi) + plane, plane * sizeof(double2),
                             cudaMemcpyDeviceToDevice, c->stream));
    return GP_OK;
}

int gp_slab_local_sums(gp_ctx *c, const void *next_first, double sums[9])
{
    if (!c || !c->slab || !sums) return fail(c, GP_EINVAL, "gp_slab_local_sums: not a z-slab or null argument");
    const long long plane = slab_plane(c);
    int rc = enqueue_observables(c);
    if (rc) return rc;
    if (next_first) {
        const double2 *last = static_cast<const double2 *>(c->psi) + (long long)(c->grid.nz - 1) * plane;
        GP_CK(c, gp::launch_slab_interface(last, next_first, plane, c->slab_part,
                                           c->slab_part + gp::kReduceBlocks, c->stream));
        GP_CK(c, cudaMemcpyAsync(c->slab_host, c->slab_part + gp::kReduceBlocks, sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
    }
    if ((rc = read_errors(c))) return rc;
    std::memcpy(sums, c->host_sums, gp::kObsWidth * sizeof(double));
    if (next_first) sums[8] += *c->slab_host;      // R_z across the interface
    return GP_OK;
}

int gp_slab_observables(gp_ctx *c, const double sums[9], gp_obs *out)
{
    if (!c || !c->slab || !sums || !out) return fail(c, GP_EINVAL, "gp_slab_observables: not a z-slab or null argument");
    finish_observables(c, sums, out);
    const double v[7] = {out->norm, out->mu, out->energy, out->rms_x, out->rms_y, out->rms_z, out->rms_r};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, GP_ENONFINITE, "gp_slab_observables: non-finite result");
    return GP_OK;
}

}  // extern "C"
