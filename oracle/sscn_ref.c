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
