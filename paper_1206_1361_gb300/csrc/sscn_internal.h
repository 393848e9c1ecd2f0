// sscn_internal.h -- shared declarations between the libgp host API and its
// CUDA kernels.  Not part of the public ABI (that is include/gp.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace gp {

// Per-axis constants of one Crank-Nicolson sweep: the line has n stored points
// (m = n - 1 unknowns at indices 1 .. n-1), kappa = kre + i kim, and the
// forward-elimination tables c'_i and mult_i (i = 1 .. m, stored 0-based).
// FP64 tables come from kappa; the complex64 tables come from the FP32
// rounding of kappa (the value the FP32 kernels multiply by), computed in
// FP64 and stored as hi + lo FP32 pairs (float4), so the FP32 elimination
// solves exactly the system whose right-hand side it forms.
// mid is the middle-row multiplier of the two-ended elimination,
// 1 / (1 + 2 kappa + kappa (c'_{k-1} + c'_{m-k})) with k = ceil(m / 2), c'_0 = 0.
struct AxisTables {
    int n = 0;
    double h = 0, kre = 0, kim = 0;
    double2 *cp64 = nullptr, *mult64 = nullptr;   // device, m entries each
    float4 *cp32 = nullptr, *mult32 = nullptr;    // device, m entries each (hi, lo)
    double2 mid64{0, 0};
    float4 mid32{0, 0, 0, 0};
    // From index conv64 (conv32) on, every FP64 (FP32) table entry equals the
    // last one: the elimination coefficients converge geometrically along a
    // constant-coefficient line, so kernels may hold c'_inf and mult_inf in
    // registers there (0-based table indices).
    int conv64 = 0, conv32 = 0;
    double2 cinf64{0, 0}, minf64{0, 0};
    float4 cinf32{0, 0, 0, 0}, minf32{0, 0, 0, 0};
    // Look-back window of the TMA path: smallest W with max|c'|^(W+1) below
    // 2^-55 (FP64) / 2^-40 (complex64); 0 if none up to 64.
    int win64 = 0, win32 = 0;
};

// Compute both table sets of one axis on the host and every derived field
// of `a` (kappa, mid, convergence, window): cp64/mult64 (FP64, from kappa)
// and cp32/mult32 (hi + lo pairs, from FP32 kappa), m entries each.
void fill_tables(AxisTables &a, int m, double kre, double kim, double2 *cp64, double2 *mult64,
                 float4 *cp32, float4 *mult32);

// A unit-modulus or real FP64 coefficient as an FP32 hi + lo pair.
float4 split_coef(double2 v);



// One sweep launch: lines are indexed by (a, b), the line's first stored point
// sits at a * stride_a + b * stride_b and its points are pstride apart.
struct SweepGeom {
    int n;               // stored points on each line
    int lines_a;         // extent of a (thread index inside the grid's x)
    int lines_b;         // extent of b (grid y)
    long long stride_a, stride_b, pstride;
};

// G, the integral of g(t) over the part [fa dt, fb dt] of step n (t = n dt)
// that one pointwise step covers: the constant G when step == nullptr, else
// for g(t) = g0 + g1 cos(omega t) read from the device step counter.  In
// real time |psi| is constant during the pointwise step, so exp(-i G |psi|^2)
// is its exact nonlinear phase for any g(t).
struct StepG {
    const long long *step = nullptr;
    double G = 0;
    double g0 = 0, g1 = 0, omega = 0, dt = 0, fa = 0, fb = 1;

#ifdef __CUDACC__
    __device__ __forceinline__ double value() const
    {
        if (!step) return G;
        const double t0 = (double)*step * dt;
        const double ta = t0 + fa * dt, tb = t0 + fb * dt;
        if (omega == 0.0) return (g0 + g1) * (tb - ta);
        return g0 * (tb - ta) + g1 * (sin(omega * tb) - sin(omega * ta)) / omega;
    }
#endif
};

// Fused potential / nonlinearity data (calcnu) of one sweep.  V is
// separable, so exp(-tau V) = P_x[i] P_y[j] P_z[k] with per-axis factor tables
// P_k[i] = exp(-tau omega_k^2 x_i^2 / 2) (tau = dt, or dt / 2 for a half step:
// real factors stored as (f, 0); tau = i dt or i dt / 2: unit complex numbers),
// computed on the host in FP64.  Only the nonlinear phase G |psi|^2 is
// evaluated per point.  The tables come in the order the sweep needs them:
// px along the sweep's lines, py and pz indexed by the line's (a, b) (x
// sweep: x; y, z.  z sweep: z; x, y.  y sweep in 2D: y; x, z).
struct NonlinArgs {
    const double2 *px = nullptr, *py = nullptr, *pz = nullptr;   // FP64 tables
    const float4 *px32 = nullptr, *py32 = nullptr, *pz32 = nullptr;   // hi + lo pairs
    // complex64 real time: phase tables theta_k = tau omega_k^2 x^2 / 2 (FP32)
    const float *tx32 = nullptr, *ty32 = nullptr, *tz32 = nullptr;
    StepG g;                         // G of the (sub)step
    const double *scale = nullptr;   // pending imaginary-time scale (device); nullptr: none
    // FP64 real-time x sweep: P_x[i] P_y[j] P_z[k] per point, laid out like psi
    // (nullptr: form it from the per-axis tables)
    const double2 *p3 = nullptr;
};

// Reduction partials of one sweep / observables pass.
struct Partials {
    double *buf = nullptr;   // device, >= blocks * width doubles
    int width = 1;
    // sweeps: weight of line a's |u|^2 (the rho_i of an axial line); nullptr: 1
    const double *line_weight = nullptr;
};

enum Precision { kC128 = 0, kC64 = 1, kCFF = 2 };

// ---- float-float form (sscn_ff.cu) ------------------------------------------
// psi as complex float-float values: per point a float4 (re_hi, im_hi, re_lo,
// im_lo), re = re_hi + re_lo (about 48 significant bits), swept with FP32
// error-free transformations on the FP32 pipe.
//
// A float-float coefficient k = kr + i ki expanded into the packed operands
// of z k = z (kr, kr) + swap(z) (-ki, ki): rh = (kr_hi, kr_hi), rl = (kr_lo,
// kr_lo), ih = (-ki_hi, ki_hi), il = (-ki_lo, ki_lo) (32 bytes).
struct FfCoef {
    float2 rh, rl, ih, il;
};
// The Crank-Nicolson tables of one axis and mode in that form: c'_i and
// mult_i (m entries each, split from the FP64 tables), the index from which
// they are constant and those constants, the back-substitution window W
// (smallest with max|c'|^(W+1) < 2^-50; 0 if none up to the chunk), and the
// coupling |kappa| = dt / (4 h^2).
struct FfAxis {
    int n = 0;
    FfCoef *cp = nullptr, *mult = nullptr;
    int conv = 0, win = 0;
    int win32 = 0;          // the window's first steps that may run in FP32
    FfCoef cinf{}, minf{};
    double k = 0;
};
// calcnu of the float-float x sweep: the factor table along the line in
// expanded form (exp(-tau omega_x^2 x_i^2 / 2)), the FP64 factor tables of
// the line's (y, z) indices, G and the pending imaginary-time scale.
struct FfNonlin {
    const FfCoef *px = nullptr;
    const double2 *py = nullptr, *pz = nullptr;
    StepG g;
    const double *scale = nullptr;
};
// Host: the float-float tables of one axis from its FP64 tables (cp64,
// mult64: m entries; conv64 / cmax: where they turn constant, their largest
// |c'|); fills `out` but not its device pointers, writes the expanded
// tables to cp / mult (host arrays of m entries).
void ff_tables(int m, const double2 *cp64, const double2 *mult64, int conv64, double cmax,
               double k, int chunk, FfAxis &out, FfCoef *cp, FfCoef *mult);
FfCoef ff_expand(double2 v);
int ff_shapes();
int ff_chunk(int shape);
int ff_blocks(int shape, const SweepGeom &g);
// Tensor map of a float-float psi for the sweep along `axis` (the layout of
// complex128: two 8-byte units per point).
cudaError_t make_ff_map(int shape, void *psi, int nx, int ny, int nz, int axis, CUtensorMap *out);
// Windowed TMA-staged float-float sweep: nl != nullptr fuses calcnu into
// the loads (x sweep); norm_out adds the FP64 sum |u|^2 per block; err
// receives bit 2 on a wait timeout.
cudaError_t launch_sweep_ff(int shape, int mode, int axis, const CUtensorMap &map,
                            const FfAxis &ax, const SweepGeom &g, const FfNonlin *nl,
                            const Partials *norm_out, int *err, cudaStream_t st);
// dst (float-float) <- split(scale * src) over count points (scale nullptr:
// 1); with reset_scale, *reset_scale <- 1 afterwards.
// complex128 psi (nx * ny * nz, device) into pairs with the Dirichlet nodes
// zeroed; src may be the caller's buffer (it is only read).
cudaError_t launch_ff_from_c128_grid(void *dst, const void *src, int nx, int ny, int nz,
                                     cudaStream_t st);
cudaError_t launch_ff_from_c128(void *dst, const void *src, long long count, const double *scale,
                                double *reset_scale, cudaStream_t st);
// Observables rows of a float-float psi (one per x-line: the FP64 row layout
// with R_k neighbour sums) and their fixed-order finish into sums[9].
// x2ff / vxff: x_i^2 and omega_x^2 x_i^2 / 2 as float-float pairs (nx each).
struct ObsArgs;
cudaError_t launch_observables_ff(const void *psi, const ObsArgs &a, const float2 *x2ff,
                                  const float2 *vxff, double *scratch, double *sums, cudaStream_t st);
// dst (complex128) <- scale * (hi + lo) over count points (scale nullptr: 1).
cudaError_t launch_ff_to_c128(void *dst, const void *src, long long count, const double *scale,
                              cudaStream_t st);

// ---- launchers (sscn_kernels.cu) -------------------------------------------
// All launchers enqueue on `st` and return the launch error (cudaSuccess if
// the launch was accepted).

// x sweep with the pending scale and the potential/nonlinear step fused in.
cudaError_t launch_sweep_x(int prec, int mode, void *psi, void *work,
                           const AxisTables &ax, const SweepGeom &g,
                           const NonlinArgs &nl, int ny, int nz,
                           const Partials *norm_out, cudaStream_t st);
// y or z sweep; norm_out != nullptr adds the FP64 sum |u|^2 per block;
// nlout != nullptr (real time, no norm) applies calcnu to every result
// before it is stored, with the tables in this sweep's order.
cudaError_t launch_sweep_yz(int prec, int mode, void *psi, void *work,
                            const AxisTables &ax, const SweepGeom &g,
                            const Partials *norm_out, cudaStream_t st,
                            const NonlinArgs *nlout = nullptr);
// calcnu as its own pass over every point (x lines; tables in x, y, z order)
// with the FP64 sums |psi|^2 into `blocks` partials: the imaginary-time
// symmetric splitting's second half step, after the renormalisation.
// wx (nullptr: 1) weights |u|^2 by the point's x index (rho_i on the axial grid).
cudaError_t launch_calcnu_pass(int prec, int mode, void *psi, int nx, int ny, int nz,
                               const NonlinArgs &nl, const Partials &norm_out, int blocks,
                               cudaStream_t st, const double *wx = nullptr);
// Fill the FP64 potential factor table p3 (nx ny nz) from the per-axis tables.
cudaError_t launch_build_pot3(void *p3, const double2 *px, const double2 *py, const double2 *pz,
                              int nx, int ny, int nz, cudaStream_t st);
// Device step counter (modulated g): set it, or add one.
cudaError_t launch_set_step(long long *step, long long value, cudaStream_t st);
cudaError_t launch_add_step(long long *step, cudaStream_t st);
int sweep_blocks(const SweepGeom &g);

// scale <- 1 / sqrt(w * sum(partials)); flags a non-finite or non-positive sum.
cudaError_t launch_norm_finish(const double *partials, int count, double w,
                               double *scale, double *norm_out, int *err,
                               cudaStream_t st);
// psi <- scale * psi over all points, then scale <- 1.
cudaError_t launch_apply_scale(int prec, void *psi, long long count,
                               double *scale, cudaStream_t st);
// Gaussian seed exp(-(gamma x^2 + nu y^2 + lambda z^2)/2), zero Dirichlet nodes.
cudaError_t launch_seed(int prec, void *psi, int nx, int ny, int nz,
                        const double h[3], const double w[3], cudaStream_t st);
// Zero the Dirichlet nodes (index 0 of each bounded axis).
cudaError_t launch_zero_boundary(int prec, void *psi, int nx, int ny, int nz,
                                 cudaStream_t st);
// FP64 sums |psi|^2 over all points into per-block partials.
cudaError_t launch_norm_partials(int prec, const void *psi, long long count,
                                 const Partials &out, int blocks, cudaStream_t st);

// Observables: the 9 FP64 sums (S0, Sx, Sy, Sz, SV, S4, Kx, Ky, Kz) of
// scale * psi, one partials row per x-line, then a fixed-order finish into
// sums[9].  FP64 grids return R_k = sum Re(psi_next conj(psi)) in place of K_k
// (the caller forms K_k = 2 S0 - 2 R_k); complex64 returns K_k.  x2/y2/z2 hold x_i^2 per axis, vx/vy/vz the potential terms
// omega_k^2 x_i^2 / 2 (device, FP64).
struct ObsArgs {
    int nx, ny, nz;
    const double *x2, *y2, *z2, *vx, *vy, *vz;
    const float *x2f, *vxf;    // FP32 roundings of x2, vx (complex64 form)
    const double *scale;   // pending scale (device)
};
// Doubles of scratch launch_observables needs for this grid.
long long obs_scratch_doubles(const ObsArgs &a);
// Observables passes that walk y-lines (complex64, float-float): threads
// along x (a multiple of 32, at most 256), blocks over (x segments, chunks of
// kObsLines lines, planes); one row of sums per block.
constexpr int kObsLines = 64;
void obs_walk_geometry(int nx, int ny, int nz, dim3 &grid, int &threads);
cudaError_t launch_observables(int prec, const void *psi, const ObsArgs &a,
                               double *scratch, double *sums, cudaStream_t st);
// Fixed-order finish of `lines` partials rows of kObsWidth doubles into sums
// (two passes through `stage`, ceil(lines / 1024) rows).
cudaError_t launch_rows_finish(const double *rows, long long lines, double *stage, double *sums,
                               cudaStream_t st);

// ---- axially symmetric psi(rho, z) (sscn_axial.cu), FP64 ---------------------
// Radial grid rho_i = (i + 1/2) h_r, i = 0 .. n_r - 1 (all unknowns, a zero
// node at i = n_r); the radial operator is tridiag(a_i, -2, c_i) / h_r^2 with
// a_i = 1 - 1/(2i+1), c_i = 1 + 1/(2i+1).  The axial grid is a Cartesian
// axis; psi[k * n_r + i].
//
// Two-ended elimination tables of (I - kappa tridiag(a, -2, c)), m = n_r
// unknowns j = 1 .. m, 0-based entry t:
//   top    (j = t + 1):  mult = 1 / (1 + 2 kappa + kappa a_j c'_{j-1}), c' = -kappa c_j mult,
//                        ka = |kappa| a_j
//   bottom (j = m - t):  mult = 1 / (1 + 2 kappa + kappa c_j e'_{j+1}), e' = -kappa a_j mult,
//                        kc = |kappa| c_j
//   middle row k = ceil(m / 2): 1 / (1 + 2 kappa + kappa (a_k c'_{k-1} + c_k e'_{k+1}))
struct RadialTables {
    const double2 *cp_top = nullptr, *mult_top = nullptr, *cp_bot = nullptr, *mult_bot = nullptr;
    const double *ka_top = nullptr, *kc_bot = nullptr;
    double2 mid{0, 0};
    double ka_mid = 0, kc_mid = 0;
};
// Host computation of those tables for kappa = kre + i kim (kre or kim zero).
void radial_tables(int m, double kre, double kim, double2 *cp_top, double2 *mult_top,
                   double2 *cp_bot, double2 *mult_bot, double *ka_top, double *kc_bot,
                   double2 *mid, double *ka_mid, double *kc_mid);
// Radial sweep of every line k (nz lines of nr points) with calcnu fused on
// the loads: nl.px = radial factor table, nl.py = axial factor table (indexed
// by the line), nl.pz = a one-entry table (1, 0).
cudaError_t launch_sweep_rho(int mode, void *psi, void *work, const RadialTables &rt, int nr,
                             int nz, const NonlinArgs &nl, cudaStream_t st);

// Segmented-window sweeps of the axial form (few, long lines).  Each line is
// cut into cores of Lc unknowns; a thread solves its core's rows extended by
// W rows on either side (zero coupling beyond the extension: the restarted
// elimination) and keeps the core.  The dropped coupling reaches the core
// damped by the product of |c'| (or |kappa a m|) over the W rows between, and
// the host picks W so that product stays below 2^-55 for every core, so the
// core rows agree with the exact solve to FP64 rounding.  The sweeps read
// `in` and write `out` (neighbouring cores read each other's rows).
struct SegWindow {
    int W = 0, Lc = 0;
    int nseg_r = 0, nseg_z = 0;         // cores per radial / axial line
    int tlen = 0;                       // radial table row: Lc + 2 W
    const double2 *cp_r = nullptr, *mult_r = nullptr;   // [nseg_r][tlen] restarted radial tables
    const double *ka_r = nullptr;       // |kappa_r| a_i, i = 0 .. nr - 1
};
// Host: restarted radial tables for cores of Lc rows and windows of W rows
// (cp, mult: nseg * (Lc + 2 W) entries each; ka: m entries).
void radial_window_tables(int m, double kre, double kim, int Lc, int W, double2 *cp, double2 *mult,
                          double *ka);
// Host: smallest window W (<= wmax, else 0) such that every core of Lc rows is
// shielded below tol from both truncations, for the radial tables of kappa.
int radial_window_width(int m, double kre, double kim, int Lc, double tol, int wmax);
// Radial: in -> out; calcnu (nl as for launch_sweep_rho) first as its own
// pass in -> pbuf (nr nz: the windows overlap, so each point's pointwise step
// is taken once), then the windowed sweep pbuf -> out; wscr (nz nseg_r W)
// holds the overlap rows.  Two launches.
cudaError_t launch_sweep_rho_win(int mode, const void *in, void *out, void *pbuf, void *wscr,
                                 const SegWindow &sw, int nr, int nz, const NonlinArgs &nl,
                                 cudaStream_t st);
// Axial: in -> out along z with the constant-coefficient tables (cp, mult of
// the z axis); nlout (real time) applies calcnu (z order: pz, px, p1) to the
// results; norm_out adds sum rho_i |u|^2 per block (rho_w).  wscr: nr nseg_z W.
cudaError_t launch_sweep_z_win(int mode, const void *in, void *out, void *wscr,
                               const SegWindow &sw, const AxisTables &az, int nr, int nz,
                               const NonlinArgs *nlout, const double *rho_w,
                               const Partials *norm_out, int *blocks, cudaStream_t st);
int sweep_rho_blocks(int nz);
// Gaussian seed exp(-(gamma rho^2 + lambda z^2) / 2), zero at k = 0.
cudaError_t launch_seed_axial(void *psi, int nr, int nz, double hr, double hz, double gamma,
                              double lambda, cudaStream_t st);
// Zero the axial Dirichlet node row k = 0.
cudaError_t launch_zero_axial(void *psi, int nr, cudaStream_t st);
// FP64 sums of rho_i |psi|^2 into `blocks` partials.
cudaError_t launch_norm_partials_axial(const void *psi, int nr, int nz, double hr,
                                       const Partials &out, int blocks, cudaStream_t st);
// Observables rows (one per line k): S0 = sum rho |psi|^2, sum rho^3 |psi|^2,
// 0, z^2 S0, sum rho V |psi|^2, sum rho |psi|^4, sum rho_{i+1/2} |psi_{i+1} - psi_i|^2,
// sum rho |psi_{k+1} - psi_k|^2, 0 (times the pending scale), then the finish.
// a.x2 / a.vx: rho^2 and gamma^2 rho^2 / 2; a.y2 / a.vy: z^2 and lambda^2 z^2 / 2.
cudaError_t launch_observables_axial(const void *psi, const ObsArgs &a, double hr,
                                     double *scratch, double *sums, cudaStream_t st);

// ---- TMA-pipelined sweeps (sscn_tma.cu) -------------------------------------
// `shape` indexes a small table of tile shapes (lines per CTA, points per
// chunk, pipeline stages); tma_shapes(prec) is its size.
int tma_shapes(int prec);
int tma_chunk(int prec, int shape);          // points per chunk C
int tma_lines(int prec, int shape);          // lines per CTA L
int tma_blocks(int prec, int shape, const SweepGeom &g);
// Tensor map of psi for the sweep along `axis`; fails (no map) when the
// layout breaks a TMA rule (complex64 rows must be a multiple of 16 bytes).
cudaError_t make_sweep_map(int prec, int shape, void *psi, int nx, int ny, int nz, int axis,
                           CUtensorMap *out);
// Windowed, TMA-staged sweep; nl != nullptr fuses calcnu: on every loaded
// point (x sweep), or with nl_at_output on every result before it is stored
// (real time, y or z sweep, no norm); norm_out adds FP64 sum |u|^2 per block;
// err receives bit 2 on a wait timeout.
cudaError_t launch_sweep_tma(int prec, int shape, int mode, int axis, const CUtensorMap &map,
                             const AxisTables &ax, const SweepGeom &g, const NonlinArgs *nl,
                             const Partials *norm_out, int *err, cudaStream_t st,
                             bool nl_at_output = false);

// Forward-elimination tables of (I - kappa L) with m unknowns, kappa = kre +
// i kim: mult_i = 1 / (1 + 2 kappa + kappa c'_{i-1}), c'_i = -kappa mult_i
// (c'_0 = 0), stored 0-based in FP64 on the host.
void host_thomas_tables(int m, double kre, double kim, double2 *cp, double2 *mult);

// One step of that recurrence, from c'_{i-1} = (pr, pi) to mult_i and c'_i,
// in real arithmetic in a fixed order with every operation rounded once:
//   z = (1 + 2 kre + kre pr - kim pi) + i (2 kim + kre pi + kim pr),
//   mult = (zr / |z|^2, -zi / |z|^2),  c' = -(kappa mult).
// The host build turns off floating-point contraction, so host and device
// (explicitly rounded intrinsics) produce the same bits.
#if defined(__CUDA_ARCH__)
#define GP_RN_MUL(a, b) __dmul_rn((a), (b))
#define GP_RN_ADD(a, b) __dadd_rn((a), (b))
#define GP_RN_SUB(a, b) __dsub_rn((a), (b))
#define GP_RN_DIV(a, b) __ddiv_rn((a), (b))
#else
#define GP_RN_MUL(a, b) ((a) * (b))
#define GP_RN_ADD(a, b) ((a) + (b))
#define GP_RN_SUB(a, b) ((a) - (b))
#define GP_RN_DIV(a, b) ((a) / (b))
#endif
#ifdef __CUDACC__
__host__ __device__
#endif
inline void thomas_step(double kre, double kim, double pr, double pi, double2 &mult, double2 &cp)
{
    const double zr = GP_RN_SUB(GP_RN_ADD(GP_RN_ADD(1.0, GP_RN_ADD(kre, kre)), GP_RN_MUL(kre, pr)),
                                GP_RN_MUL(kim, pi));
    const double zi = GP_RN_ADD(GP_RN_ADD(GP_RN_ADD(kim, kim), GP_RN_MUL(kre, pi)), GP_RN_MUL(kim, pr));
    const double d = GP_RN_ADD(GP_RN_MUL(zr, zr), GP_RN_MUL(zi, zi));
    const double mr = GP_RN_DIV(zr, d), mi = -GP_RN_DIV(zi, d);
    mult.x = mr;
    mult.y = mi;
    cp.x = -GP_RN_SUB(GP_RN_MUL(kre, mr), GP_RN_MUL(kim, mi));
    cp.y = -GP_RN_ADD(GP_RN_MUL(kre, mi), GP_RN_MUL(kim, mr));
}

// Record msg as the message gp_last_error(NULL) returns in this thread.
void set_thread_error(const char *msg);

// ---- z-slab decomposition of one grid over several GPUs (sscn_zslab.cu) -----
constexpr int kSlabMaxRanks = 8;
// Unnormalised Gaussian seed of a slab: local plane k at global plane z0 + k
// of an nzg-plane grid; local plane 0 and the x, y Dirichlet nodes zero.
cudaError_t launch_slab_seed(void *psi, int nx, int ny, int nzl, int nzg, int z0, const double h[3],
                             const double w[3], cudaStream_t st);
// saved <- psi's local planes kf and kl (two planes of `plane` points).
cudaError_t launch_slab_capture(const void *psi, void *saved, long long plane, int kf, int kl,
                                cudaStream_t st);
// bnd <- (u_loc + psi_saved) / 2 on planes kf and kl: the zero-coupling
// solution y on the slab's first and last unknown planes.
cudaError_t launch_slab_bnd(const void *psi, const void *saved, void *bnd, long long plane, int kf,
                            int kl, cudaStream_t st);
// alpha = L_{rank-1}, beta = F_{rank+1} of every z line as the combinations
// w[0 .. 2P) and w[2P .. 4P) of all ranks' bnd blocks ([P][first | last]
// [plane]), then psi[k] += 2 (s[k] alpha + t[k] beta) for local planes
// k = 1 .. nloc (spike: s then t, nloc entries each).  P = 1: nothing.
cudaError_t launch_slab_correct(void *psi, const void *bnd_all, const double2 *w,
                                const double2 *spike, int P, long long plane, int nloc,
                                cudaStream_t st);
// *out <- sum over the plane of Re(next * conj(last)) (fixed-order partials).
cudaError_t launch_slab_interface(const void *last_plane, const void *next_plane, long long plane,
                                  double *partials, double *out, cudaStream_t st);

constexpr int kObsWidth = 9;
constexpr int kReduceBlocks = 608;      // 4 x 152 SMs for grid-stride reductions

}  // namespace gp
