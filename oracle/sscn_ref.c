/*
 * sscn_ref.c -- plain FP64 CPU oracle for the split-step Crank-Nicolson (SSCN)
 * propagation of the time-dependent Gross-Pitaevskii equation
 *
 *     i dpsi/dt = [ -lap/2 + (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2)/2 + g|psi|^2 ] psi
 *
 * in a fully anisotropic harmonic trap, in real and in imaginary time (t = -i tau).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only the
 * tests, the smoke check and the benchmark's CPU-baseline / reference leg load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What the paper fixes (program summaries v, vi, xiv, xv and "Summary of
 * revisions"): the method is split-step Crank-Nicolson, propagated in real or
 * imaginary time over small steps; one step is the pointwise potential and
 * nonlinearity step (calcnu) followed by Crank-Nicolson sweeps along x, y and z
 * (calclux, calcluy, calcluz); imaginary-time runs renormalise (calcnorm); the
 * physical quantities are the chemical potential, the energy (calcmuen) and the
 * rms sizes (calcrms).  The paper prints no formula, so every step below states
 * the discretisation it uses; each one is a plain textbook definition:
 *
 *  grid     axis k keeps n_k stored points x_i = -n_k h_k / 2 + i h_k,
 *           i = 0 .. n_k - 1.  Point 0 is a zero Dirichlet node and a virtual
 *           zero node sits at i = n_k, so the unknowns are i = 1 .. n_k - 1,
 *           symmetric about x = 0.  n_z == 1 is the 2D case: z = 0, no z sweep,
 *           no z boundary.
 *  calcnu   psi <- exp(-tau (V + g |psi|^2)) psi with |psi|^2 taken before the
 *           update; tau = dt (imaginary time) or i dt (real time).
 *  calclu*  Crank-Nicolson for d psi/d tau = (1/2) d^2 psi / dx_k^2 with the
 *           3-point Laplacian L = tridiag(1, -2, 1):
 *             (I - kappa L) u = (I + kappa L) psi,  kappa = dt / (4 h_k^2)
 *           (imaginary time) or i dt / (4 h_k^2) (real time), solved on every
 *           line by forward elimination and back substitution (Thomas).
 *  calcnorm N = h_x h_y h_z sum |psi|^2 (the boundary values are zero, so the
 *           plain sum equals the trapezoid rule); imaginary time divides psi by
 *           sqrt(N) after every step.
 *  calcmuen E = W [ 1/2 sum_k K_k / h_k^2 + sum V|psi|^2 + g/2 sum |psi|^4 ] / N
 *           and mu the same with g sum |psi|^4, where W = h_x h_y h_z and K_k
 *           is the sum over every line of |psi_{i+1} - psi_i|^2 for
 *           i = 0 .. n_k - 1 (psi_{n_k} = 0): the forward differences that
 *           match the 3-point Laplacian by summation by parts.
 *  calcrms  rms_k = sqrt(sum x_k^2 |psi|^2 / sum |psi|^2), rms_r likewise
 *           with r^2 = x^2 + y^2 + z^2.
 *
 * Two extensions the paper's applications use (its cited work on a harmonic
 * modulation of the scattering length and on Faraday waves) and the paper does
 * not spell out either:
 *  g(t)     g(t) = g + g1 cos(omega t).  A pointwise step over the interval
 *           [t_a, t_b] applies the exact integral G = int g(t) dt in place of
 *           dt g: in real time |psi| is constant during that step, so
 *           psi exp(-i |psi|^2 G) solves i dpsi/dt = g(t) |psi|^2 psi exactly.
 *           Step n covers [n dt, (n + 1) dt].
 *  Strang   the symmetric splitting: a half pointwise step over the first half
 *           of the interval, the x, y, z sweeps over dt, a half pointwise step
 *           over the second half.  Second order in dt where the plain (Lie)
 *           order above is first order.  In imaginary time the state is
 *           renormalised before the second half step as well as after it:
 *           the sweeps change N by O(dt), and a nonlinear half step taken on
 *           the unnormalised state would see g scaled by that factor, which
 *           costs the fixed point its second order.
 *
 * Layout: psi[(k * n_y + j) * n_x + i], x fastest, C99 double complex.
 * Sweeps and the pointwise step may run their independent lines / points on
 * OpenMP threads (as the paper's threaded programs do); every reduction is a
 * plain serial sum in (k, j, i) order, so results do not depend on the thread
 * count.  Built with -ffp-contract=off so x86 and Arm give identical bits.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double kPi = 3.14159265358979323846;

typedef struct {
    int32_t nx, ny, nz;      /* stored points per axis; nz == 1 is 2D        */
    int32_t mode;            /* 0 = imaginary time, 1 = real time            */
    double hx, hy, hz;       /* grid spacings (hz unused when nz == 1)       */
    double dt;               /* time step                                     */
    double gamma, nu, lambda;/* trap frequencies along x, y, z               */
    double g;                /* nonlinearity                                  */
} ref_params;

/* ---------------------------------------------------------------- threads */

void ref_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ref_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------- grid */

/* Coordinate of stored point i on an axis of n points and spacing h. */
double ref_coord(int32_t n, double h, int32_t i)
{
    if (n == 1) return 0.0;
    return -0.5 * (double)n * h + (double)i * h;
}

static double cell_volume(const ref_params *p)
{
    return p->hx * p->hy * (p->nz > 1 ? p->hz : 1.0);
}

static double potential(const ref_params *p, double x, double y, double z)
{
    return 0.5 * (p->gamma * p->gamma * x * x + p->nu * p->nu * y * y +
                  p->lambda * p->lambda * z * z);
}

/* kappa of the Crank-Nicolson sweep on an axis of spacing h. */
static cplx sweep_kappa(const ref_params *p, double h)
{
    double k = p->dt / (4.0 * h * h);
    return p->mode == 1 ? k * I : k + 0.0 * I;
}

/* ------------------------------------------------------------ Thomas solve */

/*
 * Forward-elimination coefficients of (I - kappa L) for m unknowns:
 *   denom_i = (1 + 2 kappa) + kappa c'_{i-1},  c'_0 = 0,
 *   mult_i  = 1 / denom_i,   c'_i = -kappa mult_i,      i = 1 .. m.
 * Stored 0-based: cprime[i-1], mult[i-1].
 */
void ref_thomas_tables(int32_t m, double kre, double kim, cplx *cprime, cplx *mult)
{
    cplx kappa = kre + kim * I;
    cplx cprev = 0.0;
    for (int32_t i = 0; i < m; i++) {
        cplx denom = (1.0 + 2.0 * kappa) + kappa * cprev;
        mult[i] = 1.0 / denom;
        cprime[i] = -kappa * mult[i];
        cprev = cprime[i];
    }
}

/*
 * Solve (I - kappa L) u = b for m unknowns with zero values beyond both ends:
 *   -kappa u_{i-1} + (1 + 2 kappa) u_i - kappa u_{i+1} = b_i.
 * Forward: d'_i = (b_i + kappa d'_{i-1}) mult_i; back: u_m = d'_m,
 * u_i = d'_i - c'_i u_{i+1}.  u may alias b.  work needs 2 m entries.
 */
void ref_thomas_solve(int32_t m, double kre, double kim, const cplx *b, cplx *u,
                      cplx *work)
{
    cplx kappa = kre + kim * I;
    cplx *cprime = work, *mult = work + m;
    ref_thomas_tables(m, kre, kim, cprime, mult);
    cplx dprev = 0.0;
    for (int32_t i = 0; i < m; i++) {
        cplx d = (b[i] + kappa * dprev) * mult[i];
        u[i] = d;
        dprev = d;
    }
    for (int32_t i = m - 2; i >= 0; i--) u[i] = u[i] - cprime[i] * u[i + 1];
}

/*
 * One Crank-Nicolson line update in place: stored points line[0], line[s], ...
 * line[(n-1) s]; point 0 and the virtual point n are zero.  Unknowns i = 1..n-1:
 *   b_i = (1 - 2 kappa) psi_i + kappa (psi_{i-1} + psi_{i+1}),
 * then the Thomas solve with the precomputed tables.  work needs n entries.
 */
static void cn_line(int32_t n, cplx kappa, const cplx *cprime, const cplx *mult,
                    cplx *line, ptrdiff_t s, cplx *work)
{
    int32_t m = n - 1;
    cplx *d = work;                        /* d[i-1] holds d'_i */
    cplx dprev = 0.0;
    for (int32_t i = 1; i <= m; i++) {
        cplx left = (i > 1) ? line[(i - 1) * s] : 0.0;   /* Dirichlet node */
        cplx mid = line[i * s];
        cplx right = (i + 1 <= m) ? line[(i + 1) * s] : 0.0;
        cplx b = (1.0 - 2.0 * kappa) * mid + kappa * (left + right);
        cplx dd = (b + kappa * dprev) * mult[i - 1];
        d[i - 1] = dd;
        dprev = dd;
    }
    cplx u = d[m - 1];
    line[m * s] = u;
    for (int32_t i = m - 1; i >= 1; i--) {
        u = d[i - 1] - cprime[i - 1] * u;
        line[i * s] = u;
    }
}

/* --------------------------------------------------------------- the step */

/* calcnu: psi <- exp(-tau (V + g |psi|^2)) psi at every stored point. */
void ref_nonlinear(const ref_params *p, cplx *psi)
{
    const int32_t nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static)
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t j = 0; j < ny; j++) {
            double y = ref_coord(ny, p->hy, j);
            for (int32_t i = 0; i < nx; i++) {
                double x = ref_coord(nx, p->hx, i);
                size_t at = ((size_t)k * ny + j) * nx + i;
                cplx v = psi[at];
                double a = creal(v) * creal(v) + cimag(v) * cimag(v);
                double theta = p->dt * (potential(p, x, y, z) + p->g * a);
                cplx f = p->mode == 1 ? cexp(-theta * I) : exp(-theta) + 0.0 * I;
                psi[at] = f * v;
            }
        }
    }
}

/*
 * The pointwise step over part of a time step: theta = frac dt V + G |psi|^2,
 * psi <- exp(-theta) psi (imaginary time) or exp(-i theta) psi (real time),
 * where G is the integral of g over the part (frac dt g for constant g).
 */
void ref_nonlinear_part(const ref_params *p, cplx *psi, double frac, double G)
{
    const int32_t nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static)
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t j = 0; j < ny; j++) {
            double y = ref_coord(ny, p->hy, j);
            for (int32_t i = 0; i < nx; i++) {
                double x = ref_coord(nx, p->hx, i);
                size_t at = ((size_t)k * ny + j) * nx + i;
                cplx v = psi[at];
                double a = creal(v) * creal(v) + cimag(v) * cimag(v);
                double theta = frac * p->dt * potential(p, x, y, z) + G * a;
                cplx f = p->mode == 1 ? cexp(-theta * I) : exp(-theta) + 0.0 * I;
                psi[at] = f * v;
            }
        }
    }
}

/* int_{ta}^{tb} (g + g1 cos(omega t)) dt */
double ref_g_integral(double g, double g1, double omega, double ta, double tb)
{
    if (omega == 0.0) return (g + g1) * (tb - ta);
    return g * (tb - ta) + g1 * (sin(omega * tb) - sin(omega * ta)) / omega;
}

/* calclux / calcluy / calcluz: the Crank-Nicolson sweep along one axis. */
void ref_sweep(const ref_params *p, int32_t axis, cplx *psi)
{
    const int32_t nx = p->nx, ny = p->ny, nz = p->nz;
    int32_t n;
    double h;
    if (axis == 0) { n = nx; h = p->hx; }
    else if (axis == 1) { n = ny; h = p->hy; }
    else { n = nz; h = p->hz; }
    if (n < 2) return;                     /* 2D: no z sweep */
    int32_t m = n - 1;
    cplx kappa = sweep_kappa(p, h);
    cplx *cprime = malloc(sizeof(cplx) * m), *mult = malloc(sizeof(cplx) * m);
    ref_thomas_tables(m, creal(kappa), cimag(kappa), cprime, mult);
    /* the lines: (k, j) for x, (k, i) for y, (j, i) for z */
    int32_t outer = axis == 2 ? ny : nz;
    int32_t inner = axis == 0 ? ny : nx;
#pragma omp parallel
    {
        cplx *work = malloc(sizeof(cplx) * n);  /* thread-private scratch */
#pragma omp for schedule(static)
        for (int32_t a = 0; a < outer; a++) {
            for (int32_t b = 0; b < inner; b++) {
                size_t base;
                ptrdiff_t s;
                if (axis == 0) { base = ((size_t)a * ny + b) * nx; s = 1; }
                else if (axis == 1) { base = (size_t)a * ny * nx + b; s = nx; }
                else { base = (size_t)a * nx + b; s = (ptrdiff_t)nx * ny; }
                cn_line(n, kappa, cprime, mult, psi + base, s, work);
            }
        }
        free(work);
    }
    free(cprime);
    free(mult);
}

/* calcnorm: N = W sum |psi|^2, serial sum in storage order. */
double ref_norm(const ref_params *p, const cplx *psi)
{
    size_t total = (size_t)p->nx * p->ny * p->nz;
    double s = 0.0;
    for (size_t at = 0; at < total; at++)
        s += creal(psi[at]) * creal(psi[at]) + cimag(psi[at]) * cimag(psi[at]);
    return cell_volume(p) * s;
}

void ref_scale(const ref_params *p, cplx *psi, double f)
{
    size_t total = (size_t)p->nx * p->ny * p->nz;
    for (size_t at = 0; at < total; at++) psi[at] *= f;
}

/*
 * n full SSCN steps: calcnu, then the x, y, z sweeps (z skipped in 2D), then in
 * imaginary time the renormalisation psi <- psi / sqrt(N).
 */
void ref_step(const ref_params *p, cplx *psi, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; s++) {
        ref_nonlinear(p, psi);
        ref_sweep(p, 0, psi);
        ref_sweep(p, 1, psi);
        ref_sweep(p, 2, psi);
        if (p->mode == 0) ref_scale(p, psi, 1.0 / sqrt(ref_norm(p, psi)));
    }
}

/*
 * n steps starting at step index step0 (time step0 dt) with the modulated
 * g(t) = g + g1 cos(omega t) and either splitting: strang == 0 is the order of
 * ref_step with G over [t_n, t_n + dt] in place of dt g; strang == 1 is a
 * half pointwise step over [t_n, t_n + dt/2], the sweeps, (imaginary time: the
 * renormalisation), half pointwise step over [t_n + dt/2, t_n + dt], then the
 * renormalisation in imaginary time.
 */
void ref_step_ext(const ref_params *p, cplx *psi, int64_t nsteps, int64_t step0, int32_t strang,
                  double g1, double omega)
{
    for (int64_t s = 0; s < nsteps; s++) {
        double t0 = (double)(step0 + s) * p->dt;
        if (strang) {
            double th = t0 + 0.5 * p->dt, t1 = t0 + p->dt;
            ref_nonlinear_part(p, psi, 0.5, ref_g_integral(p->g, g1, omega, t0, th));
            ref_sweep(p, 0, psi);
            ref_sweep(p, 1, psi);
            ref_sweep(p, 2, psi);
            if (p->mode == 0) ref_scale(p, psi, 1.0 / sqrt(ref_norm(p, psi)));
            ref_nonlinear_part(p, psi, 0.5, ref_g_integral(p->g, g1, omega, th, t1));
        } else {
            ref_nonlinear_part(p, psi, 1.0, ref_g_integral(p->g, g1, omega, t0, t0 + p->dt));
            ref_sweep(p, 0, psi);
            ref_sweep(p, 1, psi);
            ref_sweep(p, 2, psi);
        }
        if (p->mode == 0) ref_scale(p, psi, 1.0 / sqrt(ref_norm(p, psi)));
    }
}

/*
 * Initial state: exp(-(gamma x^2 + nu y^2 + lambda z^2)/2) at the unknowns,
 * zero at the boundary nodes, normalised to N = 1.
 */
void ref_seed(const ref_params *p, cplx *psi)
{
    const int32_t nx = p->nx, ny = p->ny, nz = p->nz;
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t j = 0; j < ny; j++) {
            double y = ref_coord(ny, p->hy, j);
            for (int32_t i = 0; i < nx; i++) {
                double x = ref_coord(nx, p->hx, i);
                size_t at = ((size_t)k * ny + j) * nx + i;
                int edge = (i == 0) || (j == 0) || (nz > 1 && k == 0);
                psi[at] = edge ? 0.0
                               : exp(-0.5 * (p->gamma * x * x + p->nu * y * y +
                                             p->lambda * z * z)) + 0.0 * I;
            }
        }
    }
    ref_scale(p, psi, 1.0 / sqrt(ref_norm(p, psi)));
}

/* ------------------------------------------------------------ observables */

/*
 * The raw sums behind every observable, serial in storage order:
 * out[0] S0 = sum |psi|^2        out[1..3] sum x^2|psi|^2, y^2.., z^2..
 * out[4] SV = sum V|psi|^2       out[5]    S4 = sum |psi|^4
 * out[6..8] K_x, K_y, K_z = sums of |psi_{i+1} - psi_i|^2 along each axis
 *           over i = 0 .. n-1 with psi_n = 0 (K_z = 0 in 2D).
 */
void ref_sums(const ref_params *p, const cplx *psi, double out[9])
{
    const int32_t nx = p->nx, ny = p->ny, nz = p->nz;
    double s[9] = {0};
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t j = 0; j < ny; j++) {
            double y = ref_coord(ny, p->hy, j);
            for (int32_t i = 0; i < nx; i++) {
                double x = ref_coord(nx, p->hx, i);
                size_t at = ((size_t)k * ny + j) * nx + i;
                cplx v = psi[at];
                double a = creal(v) * creal(v) + cimag(v) * cimag(v);
                s[0] += a;
                s[1] += x * x * a;
                s[2] += y * y * a;
                s[3] += z * z * a;
                s[4] += potential(p, x, y, z) * a;
                s[5] += a * a;
                cplx nxt;
                nxt = (i + 1 < nx) ? psi[at + 1] : 0.0;
                s[6] += creal((nxt - v) * conj(nxt - v));
                nxt = (j + 1 < ny) ? psi[at + nx] : 0.0;
                s[7] += creal((nxt - v) * conj(nxt - v));
                if (nz > 1) {
                    nxt = (k + 1 < nz) ? psi[at + (size_t)nx * ny] : 0.0;
                    s[8] += creal((nxt - v) * conj(nxt - v));
                }
            }
        }
    }
    memcpy(out, s, sizeof(s));
}

/*
 * Energy pieces per particle: out[0] kinetic, out[1] potential,
 * out[2] interaction (g/2 |psi|^4), each W * sum / N.
 */
void ref_energy_parts(const ref_params *p, const cplx *psi, double out[3])
{
    double s[9];
    ref_sums(p, psi, s);
    double kin = 0.5 * (s[6] / (p->hx * p->hx) + s[7] / (p->hy * p->hy) +
                        (p->nz > 1 ? s[8] / (p->hz * p->hz) : 0.0));
    /* W * sum / (W * S0) */
    out[0] = kin / s[0];
    out[1] = s[4] / s[0];
    out[2] = 0.5 * p->g * s[5] / s[0];
}

/*
 * out[0] N, out[1] mu, out[2] E, out[3..5] rms_x, rms_y, rms_z, out[6] rms_r.
 */
void ref_observables(const ref_params *p, const cplx *psi, double out[7])
{
    double s[9];
    ref_sums(p, psi, s);
    double w = cell_volume(p);
    double n = w * s[0];
    double kin = 0.5 * (s[6] / (p->hx * p->hx) + s[7] / (p->hy * p->hy) +
                        (p->nz > 1 ? s[8] / (p->hz * p->hz) : 0.0));
    out[0] = n;
    out[1] = w * (kin + s[4] + p->g * s[5]) / n;
    out[2] = w * (kin + s[4] + 0.5 * p->g * s[5]) / n;
    out[3] = sqrt(s[1] / s[0]);
    out[4] = sqrt(s[2] / s[0]);
    out[5] = sqrt(s[3] / s[0]);
    out[6] = sqrt((s[1] + s[2] + s[3]) / s[0]);
}

/* ======================================================= axially symmetric
 *
 * The axially symmetric programs (program summaries vii, viii, xvi, xvii):
 * psi(rho, z) in a trap (gamma^2 rho^2 + lambda^2 z^2) / 2 with no angular
 * momentum,
 *     i dpsi/dt = [ -(1/2)(d^2/drho^2 + (1/rho) d/drho + d^2/dz^2) + V + g|psi|^2 ] psi.
 * The paper prints no formula; this is the discretisation used:
 *  grid    rho_i = (i + 1/2) h_r, i = 0 .. n_r - 1, all unknowns, with a zero
 *          node at i = n_r; z as the Cartesian axes (zero node at k = 0 and
 *          a virtual one at k = n_z).
 *  radial  the conservative 3-point form
 *            (L psi)_i = [rho_{i+1/2} (psi_{i+1} - psi_i) - rho_{i-1/2} (psi_i - psi_{i-1})] / (rho_i h_r^2),
 *          rho_{i +- 1/2} = rho_i +- h_r / 2, so rho_{-1/2} = 0 (no flux through
 *          the axis) and L = tridiag(a_i, -2, c_i) / h_r^2 with
 *          a_i = 1 - 1/(2i+1), c_i = 1 + 1/(2i+1).  L is self-adjoint in
 *          the inner product sum_i rho_i conj(phi_i) psi_i, so the
 *          Crank-Nicolson sweep (I - kappa L) u = (I + kappa L) psi conserves
 *          that norm in real time.
 *  norm    N = 2 pi h_r h_z sum rho_i |psi_ik|^2.
 *  E, mu   2 pi h_r h_z [ 1/2 sum rho_{i+1/2} |psi_{i+1,k} - psi_ik|^2 / h_r^2
 *          + 1/2 sum rho_i |psi_{i,k+1} - psi_ik|^2 / h_z^2 + sum rho_i V |psi|^2
 *          + (g/2 or g) sum rho_i |psi|^4 ] / N (summation by parts of L).
 *  rms     <rho^2> and <z^2> with the weights rho_i; rms_x = rms_y =
 *          sqrt(<rho^2> / 2), rms_r = sqrt(<rho^2> + <z^2>).
 * Layout psi[k * n_r + i], rho fastest.
 */
typedef struct {
    int32_t nr, nz;          /* radial points, axial points (>= 3)            */
    int32_t mode;            /* 0 imaginary, 1 real time                      */
    int32_t pad;
    double hr, hz, dt;
    double gamma, lambda;    /* radial and axial trap frequencies             */
    double g;
} ref_axial;

double ref_axial_rho(double hr, int32_t i) { return ((double)i + 0.5) * hr; }

static double axial_potential(const ref_axial *p, double r, double z)
{
    return 0.5 * (p->gamma * p->gamma * r * r + p->lambda * p->lambda * z * z);
}

/* Sub- and super-diagonal weights of the radial operator at point i. */
void ref_axial_weights(int32_t n, double *a, double *c)
{
    for (int32_t i = 0; i < n; i++) {
        double f = 1.0 / (2.0 * (double)i + 1.0);
        a[i] = 1.0 - f;
        c[i] = 1.0 + f;
    }
}

/*
 * Solve (I - kappa T) u = b with T = tridiag(a_i, -2, c_i), m unknowns and
 * zero values beyond both ends, by forward elimination and back
 * substitution: mult_i = 1 / (1 + 2 kappa + kappa a_i c'_{i-1}),
 * c'_i = -kappa c_i mult_i, d'_i = (b_i + kappa a_i d'_{i-1}) mult_i,
 * u_i = d'_i - c'_i u_{i+1}.  u may alias b; work needs 2 m entries.
 */
void ref_tridiag_solve(int32_t m, double kre, double kim, const double *a, const double *c,
                       const cplx *b, cplx *u, cplx *work)
{
    cplx kappa = kre + kim * I;
    cplx *cp = work, *d = work + m;
    cplx cprev = 0.0, dprev = 0.0;
    for (int32_t i = 0; i < m; i++) {
        cplx mult = 1.0 / (1.0 + 2.0 * kappa + kappa * a[i] * cprev);
        cp[i] = -kappa * c[i] * mult;
        d[i] = (b[i] + kappa * a[i] * dprev) * mult;
        cprev = cp[i];
        dprev = d[i];
    }
    cplx v = d[m - 1];
    u[m - 1] = v;
    for (int32_t i = m - 2; i >= 0; i--) {
        v = d[i] - cp[i] * v;
        u[i] = v;
    }
}

void ref_axial_nonlinear_part(const ref_axial *p, cplx *psi, double frac, double G)
{
    const int32_t nr = p->nr, nz = p->nz;
#pragma omp parallel for schedule(static)
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t i = 0; i < nr; i++) {
            double r = ref_axial_rho(p->hr, i);
            size_t at = (size_t)k * nr + i;
            cplx v = psi[at];
            double a = creal(v) * creal(v) + cimag(v) * cimag(v);
            double theta = frac * p->dt * axial_potential(p, r, z) + G * a;
            cplx f = p->mode == 1 ? cexp(-theta * I) : exp(-theta) + 0.0 * I;
            psi[at] = f * v;
        }
    }
}

/* Radial (axis 0) or axial (axis 1) Crank-Nicolson sweep. */
void ref_axial_sweep(const ref_axial *p, int32_t axis, cplx *psi)
{
    const int32_t nr = p->nr, nz = p->nz;
    const double h = axis == 0 ? p->hr : p->hz;
    const double kap = p->dt / (4.0 * h * h);
    const cplx kappa = p->mode == 1 ? kap * I : kap + 0.0 * I;
    /* radial lines: all n_r points are unknowns; axial lines: 1 .. n_z - 1 */
    const int32_t m = axis == 0 ? nr : nz - 1;
    const int32_t lines = axis == 0 ? nz : nr;
    double *a = malloc(sizeof(double) * m), *c = malloc(sizeof(double) * m);
    if (axis == 0) {
        ref_axial_weights(m, a, c);
    } else {
        for (int32_t i = 0; i < m; i++) a[i] = c[i] = 1.0;
    }
#pragma omp parallel
    {
        cplx *b = malloc(sizeof(cplx) * m), *work = malloc(sizeof(cplx) * 2 * m);
#pragma omp for schedule(static)
        for (int32_t l = 0; l < lines; l++) {
            /* unknown j (0-based) sits at stored index j (radial) or j + 1 (axial) */
            for (int32_t j = 0; j < m; j++) {
                size_t at, at_l = 0, at_r = 0;
                if (axis == 0) { at = (size_t)l * nr + j; at_l = at - 1; at_r = at + 1; }
                else { at = (size_t)(j + 1) * nr + l; at_l = at - nr; at_r = at + nr; }
                cplx left = j > 0 ? psi[at_l] : 0.0;
                cplx right = j + 1 < m ? psi[at_r] : 0.0;
                b[j] = (1.0 - 2.0 * kappa) * psi[at] + kappa * (a[j] * left + c[j] * right);
            }
            ref_tridiag_solve(m, creal(kappa), cimag(kappa), a, c, b, b, work);
            for (int32_t j = 0; j < m; j++) {
                size_t at = axis == 0 ? (size_t)l * nr + j : (size_t)(j + 1) * nr + l;
                psi[at] = b[j];
            }
        }
        free(b);
        free(work);
    }
    free(a);
    free(c);
}

double ref_axial_norm(const ref_axial *p, const cplx *psi)
{
    double s = 0.0;
    for (int32_t k = 0; k < p->nz; k++)
        for (int32_t i = 0; i < p->nr; i++) {
            cplx v = psi[(size_t)k * p->nr + i];
            s += ref_axial_rho(p->hr, i) * (creal(v) * creal(v) + cimag(v) * cimag(v));
        }
    return 2.0 * kPi * p->hr * p->hz * s;
}

static void axial_scale(const ref_axial *p, cplx *psi, double f)
{
    size_t total = (size_t)p->nr * p->nz;
    for (size_t at = 0; at < total; at++) psi[at] *= f;
}

/* n steps from step index step0, g(t) = g + g1 cos(omega t), plain or
 * symmetric splitting, exactly as ref_step_ext does on the Cartesian grid:
 * the radial sweep takes the place of x, the axial sweep that of y. */
void ref_axial_step_ext(const ref_axial *p, cplx *psi, int64_t nsteps, int64_t step0,
                        int32_t strang, double g1, double omega)
{
    for (int64_t s = 0; s < nsteps; s++) {
        double t0 = (double)(step0 + s) * p->dt;
        if (strang) {
            double th = t0 + 0.5 * p->dt, t1 = t0 + p->dt;
            ref_axial_nonlinear_part(p, psi, 0.5, ref_g_integral(p->g, g1, omega, t0, th));
            ref_axial_sweep(p, 0, psi);
            ref_axial_sweep(p, 1, psi);
            if (p->mode == 0) axial_scale(p, psi, 1.0 / sqrt(ref_axial_norm(p, psi)));
            ref_axial_nonlinear_part(p, psi, 0.5, ref_g_integral(p->g, g1, omega, th, t1));
        } else {
            ref_axial_nonlinear_part(p, psi, 1.0, ref_g_integral(p->g, g1, omega, t0, t0 + p->dt));
            ref_axial_sweep(p, 0, psi);
            ref_axial_sweep(p, 1, psi);
        }
        if (p->mode == 0) axial_scale(p, psi, 1.0 / sqrt(ref_axial_norm(p, psi)));
    }
}

/* exp(-(gamma rho^2 + lambda z^2) / 2), zero at the axial boundary node, N = 1. */
void ref_axial_seed(const ref_axial *p, cplx *psi)
{
    for (int32_t k = 0; k < p->nz; k++) {
        double z = ref_coord(p->nz, p->hz, k);
        for (int32_t i = 0; i < p->nr; i++) {
            double r = ref_axial_rho(p->hr, i);
            psi[(size_t)k * p->nr + i] =
                k == 0 ? 0.0 : exp(-0.5 * (p->gamma * r * r + p->lambda * z * z)) + 0.0 * I;
        }
    }
    axial_scale(p, psi, 1.0 / sqrt(ref_axial_norm(p, psi)));
}

/* out: N, mu, E, rms_x, rms_y, rms_z, rms_r (see the header of this part). */
void ref_axial_observables(const ref_axial *p, const cplx *psi, double out[7])
{
    const int32_t nr = p->nr, nz = p->nz;
    double s0 = 0, sr2 = 0, sz2 = 0, sv = 0, s4 = 0, kr = 0, kz = 0;
    for (int32_t k = 0; k < nz; k++) {
        double z = ref_coord(nz, p->hz, k);
        for (int32_t i = 0; i < nr; i++) {
            double r = ref_axial_rho(p->hr, i);
            size_t at = (size_t)k * nr + i;
            cplx v = psi[at];
            double a = creal(v) * creal(v) + cimag(v) * cimag(v);
            s0 += r * a;
            sr2 += r * r * r * a;
            sz2 += r * z * z * a;
            sv += r * axial_potential(p, r, z) * a;
            s4 += r * a * a;
            cplx nxt = i + 1 < nr ? psi[at + 1] : 0.0;
            kr += (r + 0.5 * p->hr) * creal((nxt - v) * conj(nxt - v));
            nxt = k + 1 < nz ? psi[at + nr] : 0.0;
            kz += r * creal((nxt - v) * conj(nxt - v));
        }
    }
    double w = 2.0 * kPi * p->hr * p->hz;
    double n = w * s0;
    double kin = 0.5 * (kr / (p->hr * p->hr) + kz / (p->hz * p->hz));
    out[0] = n;
    out[1] = w * (kin + sv + p->g * s4) / n;
    out[2] = w * (kin + sv + 0.5 * p->g * s4) / n;
    out[3] = sqrt(0.5 * sr2 / s0);
    out[4] = out[3];
    out[5] = sqrt(sz2 / s0);
    out[6] = sqrt((sr2 + sz2) / s0);
}
