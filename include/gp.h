/*
 * gp.h -- C ABI of libgp, a GB300 (sm_103a) implementation of the split-step
 * Crank-Nicolson (SSCN) propagation of the time-dependent Gross-Pitaevskii
 * equation in a fully anisotropic harmonic trap,
 *
 *     i dpsi/dt = [ -lap/2 + (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2)/2 + g|psi|^2 ] psi,
 *
 * in real time and in imaginary time (t = -i tau), in 3D and in 2D (nz == 1).
 *
 * The paper (program summaries v, vi, xiv, xv and "Summary of revisions") names
 * the per-step functions this library implements: calcnu (the pointwise
 * potential and nonlinearity step), calclux / calcluy / calcluz (the
 * Crank-Nicolson sweeps along x, y, z), calcnorm (normalisation), calcmuen and
 * calcrms (chemical potential, energy, rms sizes).  Discretisation:
 *
 *   grid    axis k keeps n_k stored points x_i = -n_k h_k / 2 + i h_k,
 *           i = 0 .. n_k - 1; point 0 is a zero Dirichlet node and a virtual
 *           zero node sits at i = n_k (unknowns i = 1 .. n_k - 1).  In 2D
 *           (nz == 1) z = 0 and there is no z sweep.
 *   step    psi <- exp(-tau (V + g|psi|^2)) psi, then on every x, y, z line
 *           (I - kappa L) u = (I + kappa L) psi with L = tridiag(1, -2, 1),
 *           kappa = dt / (4 h_k^2) (imaginary time, tau = dt) or
 *           i dt / (4 h_k^2) (real time, tau = i dt); imaginary time then
 *           renormalises psi to N = 1.
 *   obs     N = W sum |psi|^2 (W = h_x h_y h_z, h_x h_y in 2D);
 *           E = W [ sum_k K_k / (2 h_k^2) + sum V|psi|^2 + g/2 sum |psi|^4 ] / N,
 *           mu likewise with g sum |psi|^4, K_k the sum of squared forward
 *           differences along axis k over i = 0 .. n_k - 1; rms_k =
 *           sqrt(sum x_k^2 |psi|^2 / sum |psi|^2).
 *
 * Memory layout of psi: psi[(k * ny + j) * nx + i], x fastest, complex numbers
 * stored as interleaved (re, im): complex128 (2 x double) for GP_C128,
 * complex64 (2 x float) for GP_C64; GP_CFF exchanges complex128 through
 * gp_load / gp_store (see GP_CFF below).  Reductions always accumulate in
 * FP64.
 *
 * Conventions: every int-returning call returns GP_OK (0) or a negative GP_E*
 * code and never throws; gp_last_error() gives a message for the last failure
 * on that context.  A context owns its device memory (psi, coefficient tables,
 * reduction partials and sweep scratch), allocated in gp_create and released
 * in gp_destroy.  Host buffers passed in stay owned by the caller and are not
 * retained after the call returns.  One context must not be used from two
 * host threads at once; distinct contexts are independent.  Work is enqueued
 * on the context's CUDA stream; errors raised by the device surface at the
 * next synchronising call (gp_observables, gp_store, gp_sync).
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_ctx gp_ctx;

/* Stored points per axis; nz == 1 selects 2D.  Each of nx, ny must be >= 3,
 * nz == 1 or >= 3, and nx, ny, nz <= GP_MAX_EDGE. */
typedef struct {
    int32_t nx, ny, nz;
} gp_grid;

#define GP_MAX_EDGE 8192

enum { GP_IMAG = 0, GP_REAL = 1 };           /* propagation mode            */
/*
 * psi / sweep precision.  GP_C128: complex128 psi, FP64 arithmetic.
 * GP_C64: complex64 psi and sweeps, FP64 tables and reductions.
 * GP_CFF: the FP64-class float-float form -- psi is kept on the device as
 * float-float pairs (per point four floats: re_hi, im_hi, re_lo, im_lo,
 * re = re_hi + re_lo, about 48 significant bits) and every sweep and calcnu
 * runs in FP32 error-free arithmetic (TwoSum, FMA TwoProduct) on the FP32
 * pipe, which GB300 executes 64 times faster than FP64; tables and
 * reductions are FP64.  gp_load and gp_store exchange complex128 values;
 * gp_device_psi exposes the float-float buffer.  Cartesian grids only, the
 * TMA sweep path only (GP_OPT_SWEEP_PATH accepts GP_PATH_AUTO and
 * GP_PATH_TMA), the plain splitting only; gp_create returns GP_EINVAL when
 * an axis's back-substitution window does not fit one 8-point chunk
 * (max|c'|^9 >= 2^-50, roughly dt / (4 h^2) >= 0.02).
 */
enum { GP_C128 = 0, GP_C64 = 1, GP_CFF = 2 };

enum {
    GP_OK = 0,
    GP_EINVAL = -1,        /* bad argument: shape, spacing, dt, mode, count  */
    GP_ENOMEM = -2,        /* device or pinned host allocation failed        */
    GP_ECUDA = -3,         /* a CUDA runtime call failed                     */
    GP_ENONFINITE = -4,    /* norm or an observable came out NaN / Inf       */
    GP_ETIMEOUT = -5,      /* a bounded device wait gave up                  */
    GP_EINTERNAL = -6,     /* internal invariant violated                    */
    GP_EFULL = -7          /* a batch's memory cap cannot take the instance  */
};

/* Observables of the current state (calcnorm, calcmuen, calcrms). */
typedef struct {
    double norm, mu, energy, rms_x, rms_y, rms_z, rms_r;
    int64_t step;          /* SSCN steps taken since the last gp_load        */
    double t;              /* step * dt                                      */
} gp_obs;

/*
 * Create a context for one grid.  dx[3] = (h_x, h_y, h_z), all > 0 (h_z is
 * ignored in 2D); dt > 0; gamma, nu, lambda >= 0 are the trap frequencies; g
 * is the nonlinearity (any sign); mode GP_IMAG or GP_REAL; precision GP_C128
 * or GP_C64.  cuda_stream is a cudaStream_t to enqueue on, or NULL for a
 * stream the context creates and owns.  psi starts as zero; call gp_load.
 * On failure *out is set to NULL.
 */
int gp_create(const gp_grid *grid, const double dx[3], double dt,
              double gamma, double nu, double lambda, double g, int mode,
              int precision, void *cuda_stream, gp_ctx **out);

/*
 * Load psi.  psi points at count = nx*ny*nz interleaved complex values of the
 * context's precision, on the device (on_device = 1) or the host (0, any host
 * memory; pinned memory copies faster).  psi == NULL loads the normalised
 * anisotropic Gaussian exp(-(gamma x^2 + nu y^2 + lambda z^2)/2) instead.
 * The Dirichlet nodes (index 0 on every bounded axis) are set to zero after
 * the copy.  Resets the step counter and t to 0.  Returns GP_EINVAL if count
 * does not match the grid.
 */
int gp_load(gp_ctx *ctx, const void *psi, int64_t count, int on_device);

/*
 * Copy the current (normalised, in imaginary time) psi out to count
 * interleaved complex values of the context's precision at psi_out, on the
 * device or the host.  Synchronises the context's stream.
 */
int gp_store(gp_ctx *ctx, void *psi_out, int64_t count, int on_device);

/*
 * Change the nonlinearity and the propagation mode of the resident psi (a
 * quench: for example an imaginary-time ground state at one g continued in
 * real time at another).  Takes effect for the next gp_step.
 */
int gp_set_params(gp_ctx *ctx, double g, int mode);

/*
 * Enqueue n >= 0 SSCN steps on the context's stream and return without
 * waiting.  Each step: calcnu fused with the x sweep, the y sweep, the z
 * sweep (3D), and in imaginary time the norm reduction whose 1/sqrt(N) scale
 * is applied at the start of the next step (or by the next read).
 */
int gp_step(gp_ctx *ctx, int64_t n);

/*
 * Compute N, mu, E and the rms sizes of the current state in FP64 and copy
 * them to *out.  Synchronises the context's stream.  Returns GP_ENONFINITE
 * (and still fills *out) if any value is NaN or infinite.
 */
int gp_observables(gp_ctx *ctx, gp_obs *out);

/*
 * Per-kernel timing: run `steps` >= 1 SSCN steps without graph replay, with a
 * CUDA event on the context's stream before the first kernel of each step and
 * after each kernel, then one observables pass bracketed the same way;
 * synchronises.  ms_out[0 .. 4] receive mean milliseconds per launch of:
 * 0 the x sweep (with calcnu fused), 1 the y sweep, 2 the z sweep (0 in 2D),
 * 3 the norm finish (0 in real time), 4 the observables pass (calcmuen,
 * calcrms: kernel, finish and the 72-byte copy out).  n_out >= 5; extra
 * entries are zeroed.  The steps advance psi exactly like gp_step.
 */
int gp_time_kernels(gp_ctx *ctx, int64_t steps, double *ms_out, int n_out);

/* Kernel launches one SSCN step enqueues (the sweeps plus, in imaginary time,
 * the norm finish) into *per_step, and those one gp_observables enqueues into
 * *per_observables (either pointer may be NULL). */
int gp_launches_per_step(gp_ctx *ctx, int *per_step, int *per_observables);

/* Wait for all work enqueued on the context and report device errors. */
int gp_sync(gp_ctx *ctx);

/*
 * Device address of the context's psi buffer (valid until gp_destroy).  The
 * buffer holds psi up to a pending imaginary-time scale; call gp_store for
 * normalised values.
 */
int gp_device_psi(gp_ctx *ctx, void **dev_ptr);

/* Apply the pending imaginary-time scale 1 / sqrt(N) to the device buffer
 * (enqueued on the context's stream), so gp_device_psi holds normalised
 * values; a no-op when none is pending. */
int gp_apply_pending_scale(gp_ctx *ctx);

/*
 * One Crank-Nicolson sweep along `axis` (0 x, 1 y, 2 z; 3D only for z),
 * (I - kappa L) u = (I + kappa L) psi on every line with kappa = dt / (4 h^2)
 * (GP_IMAG) or i dt / (4 h^2) (GP_REAL), in place on psi_device: a
 * caller-owned device buffer of nx*ny*nz interleaved complex values of the
 * given precision, laid out like a context's psi.  Enqueued on cuda_stream
 * (NULL: the legacy default stream); returns without waiting.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code inside another framework's operator
 * that may only use the buffers it was given, or loops that cannot afford the
 * device-wide synchronisation of cudaMalloc / cudaFree.  It calls no device
 * allocator: the sweep's scratch and tables live in a static device array of
 * 16 MiB (+512 KiB of tables) that every GPU loading libgp holds until exit,
 * so grids above 1048576 complex128 or 2097152 complex64 points are rejected
 * with GP_EINVAL.  The first call on each device looks up the array's device
 * address; the address is kept for the life of the process, so the library
 * must not outlive a cudaDeviceReset of that device.  The coefficient tables are written into
 * the array by a small kernel on cuda_stream (nothing is staged through host
 * memory).  All calls share the one array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU race with each other.  The
 * x sweep (axis 0) runs one line per thread along contiguous x, so its
 * accesses are not coalesced and it is several times slower than the y and
 * z sweeps.  Errors: GP_EINVAL for bad arguments, GP_ECUDA if a CUDA call
 * fails; the message is in gp_last_error(NULL).
 */
int gp_sweep_noalloc(void *psi_device, const gp_grid *grid, int axis, double h,
                     double dt, int mode, int precision, void *cuda_stream);

/*
 * Z-slab decomposition of one grid over several GPUs (real time, complex128,
 * plain splitting).  The paper's largest threaded runs are real-time grids of
 * the 1000 x 1000 x 300 class; a grid beyond one GPU's memory is split along
 * z, one rank per GPU.  Rank r holds the global planes [bounds[r],
 * bounds[r+1]) of the nx * ny * nz grid (bounds[0] = 0, bounds[nranks] = nz,
 * 1 <= nranks <= 8, every rank >= 2 unknown planes: bounds[1] >= 3 and
 * bounds[r+1] - bounds[r] >= 2 above).  Its context's psi is (nz_local, ny,
 * nx) with nz_local = bounds[1] (rank 0) or bounds[r+1] - bounds[r] + 1: a
 * leading plane (the Dirichlet plane for rank 0, a zero stand-in for the
 * neighbour's last plane otherwise) and then the rank's planes.  The x and y
 * sweeps and the nonlinear step are local; the z sweep (I - kappa L) v = psi,
 * u = 2 v - psi, is a partitioned tridiagonal solve: each rank solves its own
 * block with the coupling to its neighbours cut, publishes the two boundary
 * planes of that solution, and corrects its planes after solving the
 * reduced system of all ranks' boundary values, line by line (2 (nranks - 1)
 * unknowns).  The caller moves the boundary planes between ranks (an
 * all-gather); nothing in the library talks to another GPU.
 *
 * gp_create_slab: the grid as in gp_create but global; returns GP_EINVAL for
 * an invalid partition.  The other calls of a context that apply to a slab
 * are gp_load / gp_store / gp_device_psi (the local buffer), gp_set_params
 * (real time only), gp_set_modulation, gp_set_option (plain splitting),
 * gp_sync and gp_destroy; gp_step, gp_observables, gp_time_kernels and
 * gp_autotune return GP_EINVAL.
 */
int gp_create_slab(const gp_grid *global_grid, const double dx[3], double dt, double gamma,
                   double nu, double lambda, double g, int nranks, const int *bounds, int rank,
                   void *cuda_stream, gp_ctx **out);
/* Complex128 values each rank publishes per step (2 nx ny: its first and
 * last unknown planes); the gathered buffer is nranks times that. */
int gp_slab_exchange_count(gp_ctx *ctx, int64_t *count);
/* This rank's part of the unnormalised Gaussian seed (global coordinates);
 * the caller sums the norm over ranks and applies gp_slab_scale. */
int gp_slab_seed(gp_ctx *ctx);
/* psi <- factor * psi on this rank (synchronises). */
int gp_slab_scale(gp_ctx *ctx, double factor);
/*
 * First half of one SSCN step: the nonlinear step fused into the x sweep, the
 * y sweep and the block-local z sweep, then bnd_device (2 nx ny complex128,
 * device) <- this rank's block solution on its first and last unknown
 * planes.  Enqueued on the context's stream.
 */
int gp_slab_step_begin(gp_ctx *ctx, void *bnd_device);
/*
 * Second half: bnd_all_device (device, nranks * 2 nx ny complex128, rank q's
 * planes at offset q * 2 nx ny in gp_slab_step_begin's layout) gives the
 * reduced system; this rank's planes are corrected to the coupled solution.
 * Enqueued on the context's stream after everything that wrote
 * bnd_all_device (the caller orders its collective on that stream).
 */
int gp_slab_step_end(gp_ctx *ctx, const void *bnd_all_device);
/* out_device (nx ny complex128) <- this rank's first unknown plane (the plane
 * its lower neighbour needs for the z-derivative term of the observables). */
int gp_slab_first_plane(gp_ctx *ctx, void *out_device);
/*
 * This rank's 9 observable sums (FP64; synchronises); next_first_device is
 * the next rank's gp_slab_first_plane (NULL on the last rank), for the term
 * across the interface.  The sums of all ranks add up to those of the whole
 * grid; gp_slab_observables finishes them.
 */
int gp_slab_local_sums(gp_ctx *ctx, const void *next_first_device, double sums[9]);
int gp_slab_observables(gp_ctx *ctx, const double global_sums[9], gp_obs *out);

/* Options of a context (gp_set_option / gp_get_option). */
enum {
    /* Sweep kernel: GP_PATH_AUTO picks per axis and mode; GP_PATH_EXACT is one
     * line per thread with the elimination scratch in device memory;
     * GP_PATH_TMA streams chunks of a tile of lines through shared memory with
     * TMA and back-substitutes over a window, which is only selected (and
     * only accepted) when a window W <= C (the chunk) has a truncation bound
     * max|c'|^(W+1) below 2^-40 (complex64) / 2^-55 (complex128): the
     * truncation repeats identically every step, so it is kept far below
     * one rounding. */
    GP_OPT_SWEEP_PATH = 1,
    /* Tile shape of the TMA sweep path: an index (0 .. GP_TILE_SHAPES - 1,
     * per precision) into the library's table of (lines per CTA, points per
     * chunk, pipeline stages); gp_get_option reads it back. */
    GP_OPT_TILE_SHAPE = 2,
    /* Operator splitting of one step (the paper's method is split-step
     * Crank-Nicolson; the symmetric variant is what its cited applications
     * with time-dependent interactions call for).  GP_SPLIT_LIE (default):
     * pointwise step over dt, then the x, y, z sweeps.  GP_SPLIT_STRANG: half
     * pointwise step, the sweeps, half pointwise step -- second order in dt in
     * real time, where the plain order is first order.  In imaginary time the
     * state is also renormalised before the second half step, which costs one
     * extra pass over psi per step; its fixed point stays first order in dt
     * (renormalisation does not commute with the nonlinear step) with a much
     * smaller error. */
    GP_OPT_SPLITTING = 3,
    /* 1 (default): FP64 real-time steps on the exact path read the potential
     * factor of each point from a table laid out like psi -- exp(-i dt V) for
     * the plain splitting's x sweep, exp(-i dt V / 2) for both half steps of
     * the symmetric one -- built on the first such step (one more psi-sized
     * buffer per splitting used; the sweeps are bound by the FP64 pipe, and
     * the table saves one complex multiply per point).  0: form it from the
     * per-axis tables and free the tables. */
    GP_OPT_POTENTIAL_TABLE = 4
};
/* GP_PATH_WINDOW (axial form): each line cut into cores solved in parallel,
 * each extended by a window of rows wide enough that the cut coupling reaches
 * the core below 2^-55 (the sweeps then agree with the exact solve to FP64
 * rounding); GP_PATH_AUTO takes it when a line gets at least two cores. */
/* GP_PATH_SLAB (3D Cartesian grids, nx, ny <= 256, whose xy-plane fits the
 * shared memory of one CTA -- ny (nx | 1) points of 16 (complex128) / 8
 * (complex64) bytes at most 232448 bytes -- or of a 2-CTA cluster, half the
 * rows plus a halo row each): the x and y sweeps of a step run as one pass,
 * the CTA (or cluster) holding a whole z-plane (calcnu and the x sweep on its
 * rows, the y sweep on its columns, right-hand-side form, exact elimination);
 * the z sweep takes the path GP_PATH_AUTO would.  psi crosses HBM twice per
 * step instead of three times.  Only on request (gp_set_option or
 * gp_autotune); GP_EINVAL for grids it does not fit. */
enum { GP_PATH_AUTO = 0, GP_PATH_EXACT = 1, GP_PATH_TMA = 2, GP_PATH_WINDOW = 3, GP_PATH_SLAB = 4 };
enum { GP_SPLIT_LIE = 0, GP_SPLIT_STRANG = 1 };

/*
 * Harmonic modulation of the interaction (a modulated s-wave scattering
 * length, as in the paper's cited work on parametric resonances and Faraday
 * waves): from the next step on, g(t) = g + g1 cos(omega t), with g the value
 * set by gp_create / gp_set_params and t = step * dt (the step counter is
 * reset by gp_load).  Each pointwise (sub)step over [t_a, t_b] applies the
 * exact integral of g(t) over it, which makes the real-time nonlinear phase
 * exact.  gp_observables evaluates mu and E with g(t) at the current t.
 * g1 = 0 switches it off.  GP_EINVAL for non-finite arguments.  Adds one
 * one-thread launch per step (the device step counter).
 */
int gp_set_modulation(gp_ctx *ctx, double g1, double omega);

/* Set an option; GP_EINVAL if the option or value is unknown or, for
 * GP_PATH_TMA, if some axis cannot take it.  Takes effect at the next step. */
int gp_set_option(gp_ctx *ctx, int option, int value);

/*
 * Autotune the sweep kernels for this context's grid, precision, dt and mode:
 * run `steps` SSCN steps (after one warm-up step) with every eligible (sweep
 * path, tile shape) candidate on the current state, timing each with CUDA
 * events on the context's stream, restore the state after each, and keep
 * the fastest (GP_OPT_SWEEP_PATH / GP_OPT_TILE_SHAPE are set to it).  psi,
 * the pending scale and the step counter are left as they were.  Allocates a
 * temporary copy of psi.  *path_out, *shape_out and *ms_out (mean ms per
 * step of the pick) may be NULL.  Synchronises.
 */
int gp_autotune(gp_ctx *ctx, int steps, int *path_out, int *shape_out, double *ms_out);

/* Read an option's current value into *value. */
int gp_get_option(gp_ctx *ctx, int option, int *value);

/* Number of tile shapes GP_OPT_TILE_SHAPE accepts for a precision. */
int gp_tile_shapes(int precision, int *count);

/* The sweep path each axis uses now in the current mode (GP_PATH_EXACT,
 * GP_PATH_TMA, GP_PATH_WINDOW or GP_PATH_SLAB -- the last for x and y
 * together) into path[0..2] (path[2] = 0 in 2D). */
int gp_sweep_paths(gp_ctx *ctx, int path[3]);

/*
 * Axially symmetric form (the paper's program summaries vii, viii, xvi,
 * xvii): psi(rho, z) in the trap (gamma^2 rho^2 + lambda^2 z^2) / 2, no
 * angular momentum,
 *     i dpsi/dt = [ -(1/2)(d2/drho2 + (1/rho) d/drho + d2/dz2) + V + g|psi|^2 ] psi.
 * Radial points rho_i = (i + 1/2) h_r, i = 0 .. n_r - 1 (all unknowns; zero
 * beyond the last one, no flux through the axis) with the conservative
 * 3-point radial operator, which keeps the norm 2 pi h_r h_z sum rho |psi|^2
 * in real time; axial points as a Cartesian axis (zero node at k = 0).
 * psi is FP64 (GP_C128 only), laid out psi[k * n_r + i], rho fastest.  The
 * context then takes every single-grid call: gp_load / gp_store (n_r n_z
 * values), gp_step, gp_observables (norm, mu, E; rms_x = rms_y =
 * sqrt(<rho^2> / 2), rms_z, rms_r = sqrt(<rho^2> + <z^2>)), gp_set_params,
 * GP_OPT_SPLITTING, gp_set_modulation.  The radial sweep runs the exact
 * two-ended elimination (GP_OPT_SWEEP_PATH has no TMA path here).
 * GP_EINVAL for n_r or n_z outside 3 .. 8192, h <= 0, dt <= 0, negative
 * frequencies, non-finite g or precision != GP_C128.
 */
int gp_create_axial(int nr, int nz, double hr, double hz, double dt, double gamma, double lambda,
                    double g, int mode, int precision, void *cuda_stream, gp_ctx **out);

/* Bytes of device memory gp_create_axial allocates. */
int gp_footprint_axial(int nr, int nz, int precision, size_t *bytes);

/* Bytes of device memory gp_create allocates for this grid and precision. */
int gp_footprint(const gp_grid *grid, int precision, size_t *bytes);

/*
 * Arithmetic-rate microbenchmark of the current device.  The paper has no
 * counterpart: the sweeps of the complex128 form are bound by the FP64 pipe,
 * and those of the float-float form by the FP32 pipe, so their rooflines are
 * taken against these measured rates.  kind GP_PEAK_FP64_FMA (DFMA),
 * GP_PEAK_FP32_FMA (FFMA) or GP_PEAK_FP32X2_FMA (packed two-lane FFMA2);
 * every CTA slot of the device runs `iters` >= 1 rounds of 8 independent
 * multiply-add chains per thread.  *tflops receives the best of 3 timed
 * launches (CUDA events, 2 flops per multiply-add) and *ms (may be NULL)
 * that launch's milliseconds.  Allocates 8 bytes of device memory and a
 * stream for the call; synchronises.  GP_EINVAL for a bad kind or count,
 * GP_ECUDA / GP_ENOMEM on CUDA failures (message in gp_last_error(NULL)).
 */
enum { GP_PEAK_FP64_FMA = 0, GP_PEAK_FP32_FMA = 1, GP_PEAK_FP32X2_FMA = 2 };
int gp_measure_peak(int kind, int64_t iters, double *tflops, double *ms);

/* Message for the last failure on ctx ("" if none); ctx may be NULL for the
 * last failure of a gp_create in this thread. */
const char *gp_last_error(const gp_ctx *ctx);

/* Release the context and its device memory.  NULL is a no-op. */
void gp_destroy(gp_ctx *ctx);

/* ------------------------------------------------------------------ batches
 *
 * A batch advances many independent problems -- each with its own grid
 * (edges 3 .. 512 for complex64, 3 .. 384 for complex128), spacings, trap
 * frequencies, g, dt and mode -- together: gp_batch_step runs n SSCN steps of
 * every instance in one persistent kernel launch (per 2^30 work items), whose
 * work items are (step, sweep or norm, instance, tile of 32 lines).  Each
 * instance follows the same discretisation as a context (calcnu, calclux,
 * calcluy, calcluz, calcnorm; observables calcmuen, calcrms), with the
 * elimination done exactly in shared memory, so its result does not depend
 * on which other instances share the batch.  One precision per batch;
 * reductions in FP64.  Instance memory comes from the stream-ordered
 * allocator and is charged against cap_bytes (gp_batch_footprint gives the
 * charge); gp_batch_add returns GP_EFULL when the cap cannot take it.  Slots
 * are small integers, reused after gp_batch_remove.  Errors from the device
 * surface at the next synchronising call.
 */
typedef struct gp_batch gp_batch;

int gp_batch_create(int precision, size_t cap_bytes, void *cuda_stream, gp_batch **out);
int gp_batch_footprint(const gp_grid *grid, int precision, size_t *bytes);
/* Add an instance (psi zero until gp_batch_load); *slot receives its id. */
int gp_batch_add(gp_batch *b, const gp_grid *grid, const double dx[3], double dt,
                 double gamma, double nu, double lambda, double g, int mode, int *slot);
/* As gp_load for one slot (psi NULL: the normalised Gaussian seed). */
int gp_batch_load(gp_batch *b, int slot, const void *psi, int64_t count, int on_device);
/* As gp_store for one slot; synchronises. */
int gp_batch_store(gp_batch *b, int slot, void *psi_out, int64_t count, int on_device);
/* Quench one slot: new g and mode from its next step on. */
int gp_batch_set_params(gp_batch *b, int slot, double g, int mode);
/* Advance every instance in the batch by n steps (asynchronous). */
int gp_batch_step(gp_batch *b, int64_t n);
/*
 * Budget, in nanoseconds of %globaltimer, of each dependency wait of the
 * batch's persistent kernel (a work item of one sweep waits until every item
 * of its instance's previous sweep has completed); default 2e9.  The paper
 * has no counterpart: this is failure detection for the persistent kernel.
 * A wait that exceeds its budget sets the batch's abort flag, every warp
 * leaves at its next item, and the next synchronising call (gp_batch_sync,
 * gp_batch_observables, gp_batch_store) returns GP_ETIMEOUT once; the steps
 * of that launch are then incomplete, so reload the instances before
 * stepping on.  ns = 0 makes every wait that is not satisfied at once give
 * up (used to test the path).  Takes effect at the next gp_batch_step.
 * GP_EINVAL for ns < 0.
 */
int gp_batch_set_wait_ns(gp_batch *b, int64_t ns);
/* Observables of every instance, out[slot] for slot < capacity (unused slots
 * get step = -1); synchronises. */
int gp_batch_observables(gp_batch *b, gp_obs *out, int capacity);
/*
 * Observables (the quantities of calcnorm / calcmuen / calcrms, as in
 * gp_observables) of the instances slots[0 .. count-1] only, out[i] for
 * slots[i]; synchronises.  A serving loop checks the few instances that are
 * due without paying for a pass over every instance in the batch.  Results
 * are identical to gp_batch_observables' for the same slots.  Host arrays,
 * caller-owned.  GP_EINVAL for count < 0, a NULL array with count > 0 or an
 * unused slot; errors of earlier launches as gp_batch_observables.
 */
int gp_batch_observables_of(gp_batch *b, const int *slots, int count, gp_obs *out);
/* Release one slot's memory (stream-ordered). */
int gp_batch_remove(gp_batch *b, int slot);
/* Active instances, slot table size and bytes charged against the cap. */
int gp_batch_info(gp_batch *b, int *active, int *slots, size_t *used_bytes);
int gp_batch_sync(gp_batch *b);
const char *gp_batch_last_error(const gp_batch *b);
void gp_batch_destroy(gp_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
