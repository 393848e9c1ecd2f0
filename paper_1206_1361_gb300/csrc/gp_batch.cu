// gp_batch.cu -- many independent SSCN problems (different grids, traps, g,
// dt and modes) advanced together by one persistent kernel.
//
// Work is a queue of items (step s, phase p, instance i, tile t) in that
// order: phases are the x, y and z Crank-Nicolson sweeps (calclux, calcluy,
// calcluz; calcnu fused into x) and, in imaginary time, the norm finish
// (calcnorm).  A tile is 16 or 8 lines of one instance along one axis.  Resident
// CTAs pop items from an atomic counter; before working on an item a CTA
// waits until every item of the same instance's previous phase has
// completed (a per-instance completion counter; the wait is bounded by
// %globaltimer).  Items earlier in the queue are already held by running
// CTAs, so the waits always end; instances at different phases overlap and
// no grid-wide barrier separates the sweeps.
//
// Tile solver: one warp, the tile's lines staged in shared memory (coalesced
// loads: rows for x tiles, 16-byte pieces of columns of neighbouring lines
// for y / z), each line solved in place (the right-hand side
// (1 - 2 kappa) psi_i + kappa (psi_{i-1} + psi_{i+1}) formed on the fly,
// forward elimination overwriting psi with d', back substitution overwriting
// d' with u), and the tile is written back.  Lines of fewer than 96 points:
// 16-line tiles, each line eliminated exactly from both ends by a lane pair
// (gp::solve_pair).  Longer lines: 8-line tiles, each line split into 4
// segments solved at once by 4 lanes with look-back / look-ahead windows
// (gp::solve_seg), which shortens an item's dependency chain (the latency of
// a lone instance's step) and halves the shared memory a warp holds (more
// warps resident per SM).  Lines are at most 512 points (complex64) / 384
// (complex128).  The per-instance decomposition depends only on the
// instance's own shape and coefficients, and its norm is summed in a fixed
// order, so an instance's result is bit-identical alone and in any mix.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gp.h"
#include "sscn_accum.cuh"
#include "sscn_internal.h"
#include "sscn_line.cuh"
#include "sscn_pair.cuh"
#include "sscn_seg.cuh"

namespace {

template <typename T> struct BC;
template <> struct BC<double> { using c = double2; };
template <> struct BC<float> { using c = float2; };

template <typename T> __device__ __forceinline__ typename BC<T>::c mkb(T x, T y)
{
    typename BC<T>::c r;
    r.x = x;
    r.y = y;
    return r;
}

constexpr int kPairLines = 16;     // lines per tile, two-ended pair solve
constexpr int kSegLines = 8;       // lines per tile, 4-segment solve
constexpr int kSegMinN = 96;       // edges from which an axis uses the segment solve
constexpr int kObsWidthB = gp::kObsWidth;
constexpr int kObsGroup = 16;      // x-lines per warp of the observables pass
constexpr int kMaxEdge32 = 512, kMaxEdge64 = 384;
constexpr uint64_t kWaitNs = 2000000000ull;   // default dependency-wait budget
constexpr unsigned kPollMaxNs = 512;

// Device descriptor of one active instance.
struct Inst {
    void *psi;
    int n[3];               // nx, ny, nz
    int mode;               // 0 imaginary, 1 real time
    int last_axis;          // 1 (2D) or 2 (3D)
    int tiles[3];           // tiles per axis (0 for z in 2D)
    int rows[3];            // lines per tile per axis: kPairLines or kSegLines
    int win[3];             // segment-solve window per axis (current mode)
    double kap[3];          // kappa / i (real time) or kappa (imaginary time)
    const void *cp[3], *mult[3];    // current-mode tables (Coef<T>), n - 1 entries
    int conv[3];                    // index from which the table entries are constant
    double2 cinf64[3], minf64[3];   // those constants, FP64 batches
    float4 cinf32[3], minf32[3];    // and complex64 batches (hi + lo)
    double2 mid64[3];               // middle-row multiplier of the two-ended elimination
    float4 mid32[3];
    const void *ph[3];              // current-mode potential factors (Coef<T>), n entries
    const float *th[3];             // dt omega^2 x^2 / 2 (FP32) per axis
    const double *x2[3], *v[3];     // x^2, omega^2 x^2 / 2 per axis (observables)
    const float *x2f, *vf;          // their FP32 roundings along x (complex64 observables)
    double dtg, w;
    double *scale, *norm, *partials, *obs_rows;
};

struct LaunchArgs {
    const Inst *inst;
    int N;                  // active instances
    int steps;
    long long phase_total[4];       // items per phase of one step
    long long ips;                  // items per step
    const int *pref;                // [4][N + 1] item prefix per phase
    const int *cum;                 // [N][4] items of the instance before phase p
    const int *tot;                 // [N] items of the instance per step
    unsigned long long *head;       // queue head
    int *done;                      // [N] completed items per instance
    int *err;
    int *abort_flag;
    unsigned long long wait_ns;     // budget of one dependency wait
};

// Rows of an instance's observables partials: groups of kObsGroup x-lines.
__host__ __device__ __forceinline__ long long obs_groups(int ny, int nz)
{
    return ((long long)ny * nz + kObsGroup - 1) / kObsGroup;
}

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ bool wait_done(const int *ctr, int need, const int *abort_flag, unsigned long long budget)
{
    if (ld_acquire(ctr) >= need) return true;
    const uint64_t t0 = gtime();
    unsigned ns = 32;                      // polling interval, doubled up to kPollMaxNs
    while (ld_acquire(ctr) < need) {
        if (*(volatile const int *)abort_flag) return false;
        if (gtime() - t0 >= budget) return false;
        __nanosleep(ns);
        ns = min(2 * ns, kPollMaxNs);
    }
    return true;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes):
// all copies of a tile are in flight together, then one wait.
template <int BYTES> __device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The line update of one tile row: x tiles row-major (element stride 1,
// calcnu fused into the elimination), y / z tiles column-major (stride R).
// R = kPairLines: the exact two-ended solve of a lane pair (gp::solve_pair,
// seg 0 the top lane); R = kSegLines: the 4-segment solve (gp::solve_seg,
// lane seg owning segment seg).
template <typename T, int MODE, bool NL, int R>
__device__ __forceinline__ void solve_line(const Inst &I, int axis, typename BC<T>::c *row, int n,
                                           long long line, int seg, bool active, bool norm, Acc<T> &acc)
{
    using F = typename Coef<T>::t;
    gp::PairTabs<T> tb;
    tb.mult = static_cast<const F *>(I.mult[axis]);
    tb.cp = static_cast<const F *>(I.cp[axis]);
    tb.conv = I.conv[axis];
    tb.kappa = (T)I.kap[axis];
    if constexpr (sizeof(T) == 8) {
        tb.cinf = I.cinf64[axis];
        tb.minf = I.minf64[axis];
        tb.mid = I.mid64[axis];
    } else {
        tb.cinf = I.cinf32[axis];
        tb.minf = I.minf32[axis];
        tb.mid = I.mid32[axis];
    }
    Calcnu<T, MODE> cu{};
    if (NL && active) {
        // x line: j = line % ny, k = line / ny
        const int j = (int)(line % I.n[1]), kz = (int)(line / I.n[1]);
        cu.setup(static_cast<const F *>(I.ph[0]), static_cast<const F *>(I.ph[1]),
                 static_cast<const F *>(I.ph[2]), I.th[0], I.th[1], I.th[2], j, kz, I.dtg, I.scale);
    }
    if constexpr (R == kPairLines)
        gp::solve_pair<T, MODE, NL, NL ? 1 : R>(row, 0, n, seg == 0, active, norm, acc, tb, cu);
    else
        gp::solve_seg<T, MODE, NL, NL ? 1 : R, 32 / R>(row, 0, n, seg, I.win[axis], active, norm, acc, tb, cu);
}

// Row pitch (elements) of an x tile: odd for the pair solve (lane r's column
// accesses hit distinct banks), 2 mod 4 for the segment solve (the 8 rows
// fall on distinct even bank pairs, and segments starting on points of
// opposite parity on the odd ones).
__host__ __device__ __forceinline__ int x_pitch(int n, int R)
{
    return R == kPairLines ? (n | 1) : n + ((2 - (n & 3)) & 3);
}

// Line index -> offset of its point 0 and the stride between its points.
__device__ __forceinline__ void line_geom(const Inst &I, int axis, long long L, long long &base,
                                          long long &stride)
{
    const long long nx = I.n[0], ny = I.n[1];
    if (axis == 0) { base = L * nx; stride = 1; }
    else if (axis == 1) { base = (L / nx) * nx * ny + (L % nx); stride = nx; }
    else { base = L; stride = nx * ny; }
}

// A tile of R lines in shared memory: x tiles row-major (line r at
// sm + r P, P = x_pitch), y / z tiles column-major (point c of the R lines at
// sm + R c): neighbouring y / z lines are neighbouring in memory, so a full
// tile of R consecutive lines moves as R * sizeof(C)-byte columns in 16-byte
// pieces; other y / z tiles (a row of lines ending inside the tile, a
// partial last tile, odd nx) go point by point.  Lane (r, seg) = (lane % R,
// lane / R) works on line r.
template <typename T, int R>
__device__ __forceinline__ void sweep_tile(const Inst &I, int axis, int tile, typename BC<T>::c *sm, int lane)
{
    using C = typename BC<T>::c;
    constexpr int S = 32 / R;              // lanes per line
    const int n = I.n[axis];
    const int P = x_pitch(n, R);
    const long long lines = axis == 0 ? (long long)I.n[1] * I.n[2]
                          : axis == 1 ? (long long)I.n[0] * I.n[2] : (long long)I.n[0] * I.n[1];
    const long long L0 = (long long)tile * R;
    const int rows = (int)min((long long)R, lines - L0);
    const int r = lane & (R - 1), seg = lane / R;
    const bool active = r < rows;
    C *psi = static_cast<C *>(I.psi);
    const int nx = I.n[0];                 // (kept in a register across the cp.async clobbers)
    constexpr int B = (int)sizeof(C);
    constexpr int Q = R * B / 16;          // 16-byte pieces per column
    constexpr int E = 16 / B;              // elements per piece
    long long base = 0, stride = 0, base0 = 0;
    // y / z tiles point by point: the S lanes of line r move a part each
    const int c_lo = seg * n / S, c_hi = (seg + 1) * n / S;
    bool wide = false;
    if (axis == 0) {
        for (int rr = 0; rr < rows; ++rr) {
            const C *src = psi + (L0 + rr) * nx;
            for (int c = lane; c < n; c += 32) cp_async<B>(&sm[rr * P + c], &src[c]);
        }
    } else {
        line_geom(I, axis, L0, base0, stride);
        // R lines at unit spacing, every column starting on 16 bytes
        wide = rows == R && (axis == 2 || (L0 % nx) + R <= nx) &&
               ((base0 * B) & 15) == 0 && ((stride * B) & 15) == 0;
        if (wide) {
            const C *src = psi + base0 + (lane % Q) * E;
            C *dst = sm + (lane % Q) * E;
            for (int c = lane / Q; c < n; c += 32 / Q)
                cp_async<16>(dst + c * R, src + c * stride);
        } else if (active) {
            line_geom(I, axis, L0 + r, base, stride);
            for (int c = c_lo; c < c_hi; ++c) cp_async<B>(&sm[c * R + r], &psi[base + c * stride]);
        }
    }
    // the tables the solve reads first (coefficients up to where they turn
    // constant; calcnu factors along x) into L1 while the tile's copies land:
    // the recurrences would otherwise wait on each entry in turn
    {
        const int m = n - 1, tc = min(I.conv[axis], m);
        const int tb = tc * (int)sizeof(typename Coef<T>::t);
        const char *mult = static_cast<const char *>(I.mult[axis]);
        const char *cpt = static_cast<const char *>(I.cp[axis]);
        for (int off = lane * 128; off < tb; off += 32 * 128) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(mult + off));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(cpt + off));
        }
        if (axis == 0) {
            const int pb = n * (int)sizeof(typename Coef<T>::t);
            const char *ph = static_cast<const char *>(I.ph[0]);
            for (int off = lane * 128; off < pb; off += 32 * 128)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(ph + off));
            const char *th = reinterpret_cast<const char *>(I.th[0]);
            if (th)
                for (int off = lane * 128; off < n * 4; off += 32 * 128)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(th + off));
        }
    }
    cp_async_wait_all();
    __syncwarp();
    const bool norm = I.mode == 0 && axis == I.last_axis;
    C *row = axis == 0 ? sm + r * P : sm + r;
    Acc<T> acc;
    if (axis == 0) {
        if (I.mode == 0) solve_line<T, 0, true, R>(I, axis, row, n, L0 + r, seg, active, norm, acc);
        else solve_line<T, 1, true, R>(I, axis, row, n, L0 + r, seg, active, false, acc);
    } else {
        if (I.mode == 0) solve_line<T, 0, false, R>(I, axis, row, n, L0 + r, seg, active, norm, acc);
        else solve_line<T, 1, false, R>(I, axis, row, n, L0 + r, seg, active, false, acc);
    }
    __syncwarp();
    if (axis == 0) {
        for (int rr = 0; rr < rows; ++rr) {
            C *dst = psi + (L0 + rr) * nx;
            for (int c = lane; c < n; c += 32) dst[c] = sm[rr * P + c];
        }
    } else if (wide) {
        C *dst = psi + base0 + (lane % Q) * E;
        const C *src = sm + (lane % Q) * E;
        for (int c = lane / Q; c < n; c += 32 / Q)
            *reinterpret_cast<float4 *>(dst + c * stride) =
                *reinterpret_cast<const float4 *>(src + c * R);
    } else if (active) {
        for (int c = c_lo; c < c_hi; ++c) psi[base + c * stride] = sm[c * R + r];
    }
    if (norm) {
        const double v = warp_sum_d(acc.get());
        if (lane == 0) I.partials[tile] = v;
    }
}

// calcnorm of one instance: FP64 sum of its last-sweep tile partials in
// fixed order, scale <- 1 / sqrt(N).
__device__ void norm_item(const Inst &I, int lane, int *err)
{
    const int tiles = I.tiles[I.last_axis];
    // four interleaved FP64 chains per lane (a dependent FP64 add is slow on
    // GB300), combined in a fixed order
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int t = lane;
    for (; t + 96 < tiles; t += 128) {
        v0 += I.partials[t];
        v1 += I.partials[t + 32];
        v2 += I.partials[t + 64];
        v3 += I.partials[t + 96];
    }
    for (; t < tiles; t += 32) v0 += I.partials[t];
    const double v = warp_sum_d((v0 + v1) + (v2 + v3));
    if (lane == 0) {
        const double nrm = I.w * v;
        *I.norm = nrm;
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            atomicOr(err, 1);
            *I.scale = 1.0;
        } else {
            *I.scale = 1.0 / sqrt(nrm);
        }
    }
}

// The instance owning item r of a phase: the largest a with pr[a] <= r
// (pr non-decreasing, pr[0] = 0 <= r < pr[N]).  The warp samples up to 32
// entries per round and a ballot picks the last one <= r (a prefix, pr being
// sorted), so a search over N instances takes ceil(log32(N + 1)) dependent
// loads instead of log2(N).
__device__ __forceinline__ int find_instance(const int *pr, int N, int r, int lane)
{
    int lo = 0, span = N + 1;              // the answer lies in [lo, lo + span)
    for (;;) {
        const int S = span > 32 ? (span + 31) >> 5 : 1;
        const int idx = lo + lane * S;
        const bool ok = idx < lo + span && pr[idx] <= r;
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        const int j = 31 - __clz(bal);     // lane 0 always votes yes: pr[lo] <= r
        const int nlo = lo + j * S;
        if (S == 1) return nlo;
        span = min(S, lo + span - nlo);
        lo = nlo;
    }
}

template <typename T>
__global__ void __launch_bounds__(32) k_batch_steps(const __grid_constant__ LaunchArgs A)
{
    using C = typename BC<T>::c;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int lane = threadIdx.x;
    const long long total = A.ips * A.steps;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(A.head, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((long long)it >= total) break;
        if (*(volatile const int *)A.abort_flag) break;
        const int s = (int)((long long)it / A.ips);
        long long r = (long long)it - (long long)s * A.ips;
        int p = 0;
        // (constant indices: a dynamically indexed kernel-parameter array
        // would be copied to local memory)
        if (r >= A.phase_total[0]) {
            r -= A.phase_total[0];
            ++p;
            if (r >= A.phase_total[1]) {
                r -= A.phase_total[1];
                ++p;
                if (r >= A.phase_total[2]) {
                    r -= A.phase_total[2];
                    ++p;
                }
            }
        }
        const int *pr = A.pref + p * (A.N + 1);
        const int i = find_instance(pr, A.N, (int)r, lane), tile = (int)(r - pr[i]);
        const Inst &I = A.inst[i];
        // its descriptor into L1 while the dependency wait runs
        if (lane * 128 < (int)sizeof(Inst))
            asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char *>(&I) + lane * 128));
        const int need = s * A.tot[i] + A.cum[i * 4 + p];
        int ok = 1;
        if (lane == 0) ok = wait_done(&A.done[i], need, A.abort_flag, A.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                atomicOr(A.err, 2);
                atomicExch(A.abort_flag, 1);
            }
            break;
        }
        // lane 0's acquire, then the warp barrier (which orders memory among
        // its lanes), make the previous phase's stores visible to every lane
        __syncwarp();
        if (p < 3) {
            if (I.rows[p] == kSegLines) sweep_tile<T, kSegLines>(I, p, tile, sm, lane);
            else sweep_tile<T, kPairLines>(I, p, tile, sm, lane);
        }
        else norm_item(I, lane, A.err);
        // the barrier orders every lane's stores before lane 0's release,
        // which carries them (cumulatively) to the waiting warps
        __syncwarp();
        if (lane == 0) red_release_add(&A.done[i], 1);
    }
}

// ---------------------------------------------------------------- observables

// One warp per group of kObsGroup consecutive x-lines of the instances
// inst[idx[0 .. M-1]] (grp_pref: prefix of their groups), the lanes across
// x: the sums of the observables pass (|psi|^2, x^2 |psi|^2 per axis,
// V |psi|^2, |psi|^4 and the forward-difference kinetic terms) over the
// group into one row of I.obs_rows.  The per-line factors (y^2, z^2 and
// V_y + V_z) multiply each lane's partial |psi|^2 of the line in FP64; a
// warp reduces once per group, not once per line.
template <typename T>
__global__ void __launch_bounds__(256)
k_batch_obs(const Inst *inst, const int *idx, const long long *grp_pref, int N)
{
    using C = typename BC<T>::c;
    const int lane = threadIdx.x & 31;
    const long long g = (long long)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g >= grp_pref[N]) return;
    int lo = 0, hi = N;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (grp_pref[mid] <= g) lo = mid;
        else hi = mid;
    }
    const Inst &I = inst[idx[lo]];
    const long long grp = g - grp_pref[lo];
    const int nx = I.n[0], ny = I.n[1], nz = I.n[2];
    const long long l0 = grp * kObsGroup, l1 = min((long long)ny * nz, l0 + kObsGroup);
    const long long plane = (long long)nx * ny;
    const C *psi = static_cast<const C *>(I.psi);
    const C zero = mkb<T>((T)0, (T)0);
    Acc<T> sx, svx, s4, kx, ky, kz;
    double s0 = 0.0, fy = 0.0, fz = 0.0, fv = 0.0;
    const T *x2 = sizeof(T) == 8 ? (const T *)I.x2[0] : (const T *)I.x2f;
    const T *vx = sizeof(T) == 8 ? (const T *)I.v[0] : (const T *)I.vf;
    const double *x2y = I.x2[1], *x2z = I.x2[2], *vy = I.v[1], *vz = I.v[2];
    for (long long line = l0; line < l1; ++line) {
        const int j = (int)(line % ny), k = (int)(line / ny);
        const C *row = psi + line * nx;
        const bool has_y = j + 1 < ny, has_z = k + 1 < nz;
        Acc<T> ls;
        for (int i = lane; i < nx; i += 32) {
            const C v = row[i];
            const T am = fma(v.x, v.x, v.y * v.y);
            ls.add(am);
            sx.add_prod(x2[i], am);
            svx.add_prod(vx[i], am);
            s4.add_prod(am, am);
            const C nb = (i + 1 < nx) ? row[i + 1] : zero;
            kx.add_sq2(nb.x - v.x, nb.y - v.y);
            const C ny_ = has_y ? row[i + nx] : zero;
            ky.add_sq2(ny_.x - v.x, ny_.y - v.y);
            if (nz > 1) {
                const C nz_ = has_z ? row[i + plane] : zero;
                kz.add_sq2(nz_.x - v.x, nz_.y - v.y);
            }
        }
        const double p = ls.get();
        s0 += p;
        fy = fma(x2y[j], p, fy);
        fz = fma(x2z[k], p, fz);
        fv = fma(vy[j] + vz[k], p, fv);
    }
    double rx, rv, r4, qx, qy, qz;
    if constexpr (sizeof(T) == 4) {
        rx = warp_sum_comp(sx.s, sx.c);
        rv = warp_sum_comp(svx.s, svx.c);
        r4 = warp_sum_comp(s4.s, s4.c);
        qx = warp_sum_comp(kx.s, kx.c);
        qy = warp_sum_comp(ky.s, ky.c);
        qz = warp_sum_comp(kz.s, kz.c);
    } else {
        rx = warp_sum_d(sx.get());
        rv = warp_sum_d(svx.get());
        r4 = warp_sum_d(s4.get());
        qx = warp_sum_d(kx.get());
        qy = warp_sum_d(ky.get());
        qz = warp_sum_d(kz.get());
    }
    const double r0 = warp_sum_d(s0), ry = warp_sum_d(fy), rz = warp_sum_d(fz), rvv = warp_sum_d(fv);
    if (lane == 0) {
        const double sc = *I.scale, s2 = sc * sc;
        double *out = I.obs_rows + grp * kObsWidthB;
        out[0] = s2 * r0;
        out[1] = s2 * rx;
        out[2] = s2 * ry;
        out[3] = s2 * rz;
        out[4] = s2 * (rv + rvv);
        out[5] = s2 * s2 * r4;
        out[6] = s2 * qx;
        out[7] = s2 * qy;
        out[8] = s2 * qz;
    }
}

// One block per instance inst[idx[i]]: its rows summed in a fixed order into
// sums[i][9].
__global__ void __launch_bounds__(256) k_batch_obs_finish(const Inst *inst, const int *idx, double *sums)
{
    __shared__ double red[8];
    const Inst &I = inst[idx[blockIdx.x]];
    const long long rows = obs_groups(I.n[1], I.n[2]);
    for (int q = 0; q < kObsWidthB; ++q) {
        double v = 0.0;
        for (long long r = threadIdx.x; r < rows; r += blockDim.x) v += I.obs_rows[r * kObsWidthB + q];
        v = warp_sum_d(v);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
            t = warp_sum_d(t);
            if (threadIdx.x == 0) sums[(long long)blockIdx.x * kObsWidthB + q] = t;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void k_batch_apply_scale(typename BC<T>::c *psi, long long count, double *scale)
{
    const T s = (T)*scale;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        auto v = psi[p];
        v.x *= s;
        v.y *= s;
        psi[p] = v;
    }
}

__global__ void k_batch_set_one(double *x) { *x = 1.0; }

}  // namespace

// ====================================================================== host

struct gp_batch_slot {
    bool used = false;
    gp_grid grid{};
    double h[3]{}, dt = 0, w[3]{}, g = 0;
    int mode = 0;
    int64_t step = 0;
    bool scale_pending = false;
    void *psi = nullptr;            // device, points * elem
    unsigned char *aux = nullptr;   // device: tables, scalars, partials, rows
    size_t bytes = 0;               // footprint charged against the cap
    // device pointers into aux
    void *cp[2][3]{}, *mult[2][3]{}, *ph[2][3]{};
    double *x2[3]{}, *v[3]{};
    float *th[3]{};
    float *x2f = nullptr, *vf = nullptr;
    double *scale = nullptr, *norm = nullptr, *partials = nullptr, *obs_rows = nullptr;
    gp::AxisTables conv[2][3];      // convergence fields per mode/axis (host)
    int win[2][3]{};                // segment-solve windows per mode/axis
};

struct gp_batch {
    int prec = GP_C64;
    size_t cap = 0, used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<gp_batch_slot> slots;
    bool dirty = true;
    // launch structures
    std::vector<int> active;        // slot ids in launch order
    Inst *d_inst = nullptr;
    int *d_ints = nullptr;          // pref | cum | tot | done | err | abort
    size_t ints_cap = 0;
    unsigned long long *d_head = nullptr;
    int *d_err = nullptr;           // error bits, abort flag
    double *d_sums = nullptr;
    size_t inst_cap = 0;
    double *h_sums = nullptr;       // pinned
    // observables of a subset: M + 1 line prefixes then M active indices,
    // staged in pinned memory and copied to the device in one piece
    unsigned char *d_sub = nullptr, *h_sub = nullptr;
    int *h_err = nullptr;           // pinned
    unsigned long long wait_ns = kWaitNs;
    LaunchArgs args{};
    size_t smem = 0;
    int grid = 0;
    std::string last_error;
};

namespace {

int bfail(gp_batch *b, int code, const std::string &msg)
{
    if (b) b->last_error = msg;
    else gp::set_thread_error(msg.c_str());
    return code;
}

#define GP_BCK(b, call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

size_t elem(int prec) { return prec == GP_C128 ? 16 : 8; }

bool batch_grid_ok(const gp_grid *g, int prec)
{
    const int mx = prec == GP_C128 ? kMaxEdge64 : kMaxEdge32;
    auto ok = [&](int n) { return n >= 3 && n <= mx; };
    return g && ok(g->nx) && ok(g->ny) && (g->nz == 1 || ok(g->nz));
}

int edge_of(const gp_grid &g, int k) { return k == 0 ? g.nx : (k == 1 ? g.ny : g.nz); }
int axes_of(const gp_grid &g) { return g.nz > 1 ? 3 : 2; }

long long lines_of(const gp_grid &g, int axis)
{
    const long long nx = g.nx, ny = g.ny, nz = g.nz;
    return axis == 0 ? ny * nz : axis == 1 ? nx * nz : nx * ny;
}

// Lines per tile of an axis with n points per line (a function of the
// shape alone, so tile counts do not change with the mode).
int tile_rows(int n) { return n >= kSegMinN ? kSegLines : kPairLines; }

int tiles_of(const gp_grid &g, int axis)
{
    if (axis >= axes_of(g)) return 0;
    const int R = tile_rows(edge_of(g, axis));
    return (int)((lines_of(g, axis) + R - 1) / R);
}

// Shared-memory elements of one tile along an axis.
size_t tile_elems(const gp_grid &g, int axis)
{
    const int n = edge_of(g, axis), R = tile_rows(n);
    return (size_t)R * (axis == 0 ? x_pitch(n, R) : n);
}

// Window of the segment solve: the least W with cmax^(W+1) < eps (cmax the
// largest |c'_i| of the axis), or a width past any line (exact) if there is
// none below 1024.
int seg_window(double cmax, double eps)
{
    double p = cmax;
    for (int w = 0; w < 1024; ++w) {
        if (p < eps) return w;
        p *= cmax;
    }
    return 1 << 20;
}

// Layout of a slot's aux block (byte offsets), 256-byte aligned pieces.
struct AuxLayout {
    size_t cp[2][3], mult[2][3], ph[2][3], th[3], x2[3], v[3], x2f, vf, scale, norm, partials, rows, total;
};

AuxLayout aux_layout(const gp_grid &g, int prec)
{
    AuxLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~size_t(255);
        return at;
    };
    const size_t e = 16;                   // double2 or float4 (hi + lo) coefficients
    (void)prec;
    for (int mode = 0; mode < 2; ++mode)
        for (int k = 0; k < 3; ++k) {
            const size_t n = edge_of(g, k);
            L.cp[mode][k] = take(n * e);
            L.mult[mode][k] = take(n * e);
            L.ph[mode][k] = take(n * e);
        }
    for (int k = 0; k < 3; ++k) {
        L.th[k] = take(edge_of(g, k) * sizeof(float));
        L.x2[k] = take(edge_of(g, k) * sizeof(double));
        L.v[k] = take(edge_of(g, k) * sizeof(double));
    }
    L.x2f = take(edge_of(g, 0) * sizeof(float));
    L.vf = take(edge_of(g, 0) * sizeof(float));
    L.scale = take(sizeof(double));
    L.norm = take(sizeof(double));
    L.partials = take((size_t)std::max(1, tiles_of(g, axes_of(g) - 1)) * sizeof(double));
    L.rows = take((size_t)lines_of(g, 0) * gp::kObsWidth * sizeof(double));
    L.total = off;
    return L;
}

size_t slot_bytes(const gp_grid &g, int prec)
{
    return (size_t)g.nx * g.ny * g.nz * elem(prec) + aux_layout(g, prec).total;
}

double coord_b(int n, double h, int i) { return n == 1 ? 0.0 : -0.5 * n * h + i * h; }

// Upload tables, potential factors and observables tables of a slot.
int upload_slot(gp_batch *b, gp_batch_slot &s)
{
    const AuxLayout L = aux_layout(s.grid, b->prec);
    const int nd = axes_of(s.grid);
    std::vector<unsigned char> host(L.total, 0);
    auto put = [&](size_t off, const void *src, size_t bytes) { std::memcpy(host.data() + off, src, bytes); };
    for (int mode = 0; mode < 2; ++mode)
        for (int k = 0; k < 3; ++k) {
            const int n = edge_of(s.grid, k), m = n - 1;
            if (k < nd) {
                const double kap = s.dt / (4.0 * s.h[k] * s.h[k]);
                std::vector<double2> cp(m), mult(m);
                std::vector<float4> c32(m), m32(m);
                gp::AxisTables &a = s.conv[mode][k];
                gp::fill_tables(a, m, mode == 0 ? kap : 0.0, mode == 0 ? 0.0 : kap, cp.data(), mult.data(),
                                c32.data(), m32.data());
                // dropped window terms below the storage rounding: 2^-32
                // (complex64, 24-bit significands), 2^-56 (complex128)
                double cmax = 0.0;
                for (int i = 0; i < m; ++i) cmax = std::max(cmax, std::hypot(cp[i].x, cp[i].y));
                s.win[mode][k] = seg_window(cmax, std::ldexp(1.0, b->prec == GP_C128 ? -56 : -32));
                if (b->prec == GP_C128) {
                    put(L.cp[mode][k], cp.data(), m * sizeof(double2));
                    put(L.mult[mode][k], mult.data(), m * sizeof(double2));
                } else {
                    put(L.cp[mode][k], c32.data(), m * sizeof(float4));
                    put(L.mult[mode][k], m32.data(), m * sizeof(float4));
                }
            }
            std::vector<double2> ph(n);
            for (int i = 0; i < n; ++i) {
                const double x = coord_b(n, s.h[k], i);
                const double th = s.dt * 0.5 * s.w[k] * s.w[k] * x * x;
                ph[i] = mode == 0 ? make_double2(std::exp(-th), 0.0) : make_double2(std::cos(th), -std::sin(th));
            }
            if (b->prec == GP_C128) put(L.ph[mode][k], ph.data(), n * sizeof(double2));
            else {
                std::vector<float4> p32(n);
                for (int i = 0; i < n; ++i) p32[i] = gp::split_coef(ph[i]);
                put(L.ph[mode][k], p32.data(), n * sizeof(float4));
            }
        }
    for (int k = 0; k < 3; ++k) {
        const int n = edge_of(s.grid, k);
        std::vector<double> x2(n), v(n);
        for (int i = 0; i < n; ++i) {
            const double x = coord_b(n, s.h[k], i);
            x2[i] = x * x;
            v[i] = 0.5 * s.w[k] * s.w[k] * x * x;
        }
        put(L.x2[k], x2.data(), n * sizeof(double));
        put(L.v[k], v.data(), n * sizeof(double));
        std::vector<float> th(n);
        for (int i = 0; i < n; ++i) th[i] = (float)(s.dt * v[i]);
        put(L.th[k], th.data(), n * sizeof(float));
        if (k == 0) {
            std::vector<float> x2f(x2.begin(), x2.end()), vf(v.begin(), v.end());
            put(L.x2f, x2f.data(), n * sizeof(float));
            put(L.vf, vf.data(), n * sizeof(float));
        }
    }
    const double one = 1.0;
    put(L.scale, &one, sizeof(double));
    GP_BCK(b, cudaMemcpyAsync(s.aux, host.data(), L.total, cudaMemcpyHostToDevice, b->stream));
    GP_BCK(b, cudaStreamSynchronize(b->stream));       // `host` goes out of scope
    for (int mode = 0; mode < 2; ++mode)
        for (int k = 0; k < 3; ++k) {
            s.cp[mode][k] = s.aux + L.cp[mode][k];
            s.mult[mode][k] = s.aux + L.mult[mode][k];
            s.ph[mode][k] = s.aux + L.ph[mode][k];
        }
    for (int k = 0; k < 3; ++k) {
        s.x2[k] = reinterpret_cast<double *>(s.aux + L.x2[k]);
        s.v[k] = reinterpret_cast<double *>(s.aux + L.v[k]);
        s.th[k] = reinterpret_cast<float *>(s.aux + L.th[k]);
    }
    s.x2f = reinterpret_cast<float *>(s.aux + L.x2f);
    s.vf = reinterpret_cast<float *>(s.aux + L.vf);
    s.scale = reinterpret_cast<double *>(s.aux + L.scale);
    s.norm = reinterpret_cast<double *>(s.aux + L.norm);
    s.partials = reinterpret_cast<double *>(s.aux + L.partials);
    s.obs_rows = reinterpret_cast<double *>(s.aux + L.rows);
    return GP_OK;
}

Inst make_inst(const gp_batch_slot &s, int prec)
{
    Inst I{};
    I.psi = s.psi;
    I.n[0] = s.grid.nx;
    I.n[1] = s.grid.ny;
    I.n[2] = s.grid.nz;
    I.mode = s.mode;
    I.last_axis = axes_of(s.grid) - 1;
    for (int k = 0; k < 3; ++k) {
        I.tiles[k] = tiles_of(s.grid, k);
        I.rows[k] = tile_rows(edge_of(s.grid, k));
        I.win[k] = s.win[s.mode][k];
        I.kap[k] = k < axes_of(s.grid) ? s.dt / (4.0 * s.h[k] * s.h[k]) : 0.0;
        I.cp[k] = s.cp[s.mode][k];
        I.mult[k] = s.mult[s.mode][k];
        const gp::AxisTables &a = s.conv[s.mode][k];
        I.conv[k] = prec == GP_C128 ? a.conv64 : a.conv32;
        I.cinf64[k] = a.cinf64;
        I.minf64[k] = a.minf64;
        I.cinf32[k] = a.cinf32;
        I.minf32[k] = a.minf32;
        I.mid64[k] = a.mid64;
        I.mid32[k] = a.mid32;
        I.ph[k] = s.ph[s.mode][k];
        I.th[k] = s.th[k];
        I.x2[k] = s.x2[k];
        I.v[k] = s.v[k];
    }
    I.x2f = s.x2f;
    I.vf = s.vf;
    I.dtg = s.dt * s.g;
    I.w = s.h[0] * s.h[1] * (s.grid.nz > 1 ? s.h[2] : 1.0);
    I.scale = s.scale;
    I.norm = s.norm;
    I.partials = s.partials;
    I.obs_rows = s.obs_rows;
    return I;
}

// Bytes of the subset staging block for up to cap instances.
size_t sub_bytes(size_t cap) { return (cap + 1) * sizeof(long long) + cap * sizeof(int); }

int ensure_capacity(gp_batch *b, size_t n_inst)
{
    if (n_inst <= b->inst_cap && b->d_inst) return GP_OK;
    const size_t cap = std::max<size_t>(64, n_inst * 2);
    if (b->d_inst) cudaFreeAsync(b->d_inst, b->stream);
    if (b->d_sub) cudaFreeAsync(b->d_sub, b->stream);
    if (b->d_sums) cudaFreeAsync(b->d_sums, b->stream);
    if (b->h_sums || b->h_sub) {
        cudaStreamSynchronize(b->stream);
        if (b->h_sums) cudaFreeHost(b->h_sums);
        if (b->h_sub) cudaFreeHost(b->h_sub);
        b->h_sums = nullptr;
        b->h_sub = nullptr;
    }
    GP_BCK(b, cudaMallocAsync((void **)&b->d_inst, cap * sizeof(Inst), b->stream));
    GP_BCK(b, cudaMallocAsync((void **)&b->d_sub, sub_bytes(cap), b->stream));
    GP_BCK(b, cudaMallocAsync((void **)&b->d_sums, cap * gp::kObsWidth * sizeof(double), b->stream));
    GP_BCK(b, cudaMallocHost((void **)&b->h_sums, cap * gp::kObsWidth * sizeof(double)));
    GP_BCK(b, cudaMallocHost((void **)&b->h_sub, sub_bytes(cap)));
    b->inst_cap = cap;
    return GP_OK;
}

// Rebuild the instance descriptors and the item prefix arrays.
int prepare(gp_batch *b)
{
    if (!b->dirty) return GP_OK;
    b->active.clear();
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (b->slots[i].used) b->active.push_back((int)i);
    const int N = (int)b->active.size();
    if (N == 0) {
        b->dirty = false;
        return GP_OK;
    }
    int rc = ensure_capacity(b, N);
    if (rc) return rc;
    std::vector<Inst> inst(N);
    std::vector<int> pref(4 * (N + 1), 0), cum(4 * N, 0), tot(N, 0);
    long long ptot[4] = {0, 0, 0, 0};
    size_t max_elems = 1;
    for (int a = 0; a < N; ++a) {
        const gp_batch_slot &s = b->slots[b->active[a]];
        inst[a] = make_inst(s, b->prec);
        int items[4];
        for (int k = 0; k < 3; ++k) items[k] = tiles_of(s.grid, k);
        items[3] = s.mode == 0 ? 1 : 0;
        int c = 0;
        for (int p = 0; p < 4; ++p) {
            cum[a * 4 + p] = c;
            c += items[p];
            pref[p * (N + 1) + a + 1] = pref[p * (N + 1) + a] + items[p];
            ptot[p] += items[p];
        }
        tot[a] = c;
        for (int k = 0; k < axes_of(s.grid); ++k) max_elems = std::max(max_elems, tile_elems(s.grid, k));
    }
    const size_t nints = pref.size() + cum.size() + tot.size() + N;
    if (nints > b->ints_cap) {
        if (b->d_ints) cudaFreeAsync(b->d_ints, b->stream);
        b->ints_cap = nints * 2;
        GP_BCK(b, cudaMallocAsync((void **)&b->d_ints, b->ints_cap * sizeof(int), b->stream));
    }
    std::vector<int> ints;
    ints.insert(ints.end(), pref.begin(), pref.end());
    ints.insert(ints.end(), cum.begin(), cum.end());
    ints.insert(ints.end(), tot.begin(), tot.end());
    GP_BCK(b, cudaMemcpyAsync(b->d_inst, inst.data(), N * sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
    GP_BCK(b, cudaMemcpyAsync(b->d_ints, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    GP_BCK(b, cudaStreamSynchronize(b->stream));
    LaunchArgs &A = b->args;
    A.inst = b->d_inst;
    A.N = N;
    for (int p = 0; p < 4; ++p) A.phase_total[p] = ptot[p];
    A.ips = ptot[0] + ptot[1] + ptot[2] + ptot[3];
    A.pref = b->d_ints;
    A.cum = A.pref + pref.size();
    A.tot = A.cum + cum.size();
    A.done = const_cast<int *>(A.tot) + N;
    A.err = b->d_err;
    A.abort_flag = b->d_err + 1;
    A.head = b->d_head;
    b->smem = max_elems * elem(b->prec);
    int per_sm = 0, sms = 0, dev = 0;
    GP_BCK(b, cudaGetDevice(&dev));
    GP_BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (b->prec == GP_C128) {
        GP_BCK(b, cudaFuncSetAttribute(k_batch_steps<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
        GP_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_steps<double>, 32, b->smem));
    } else {
        GP_BCK(b, cudaFuncSetAttribute(k_batch_steps<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
        GP_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_steps<float>, 32, b->smem));
    }
    // persistent grid: every resident warp, but no more than the widest
    // phase.  Warps beyond that would only hold later items and poll their
    // dependency counters, which with a few small instances left (the tail
    // of a batch of solves) crowds the L2 around the counters that the
    // working warps update (a lone 128 x 128 x 32 instance: 83 us per step
    // with twice the widest phase, 66 us with once).
    long long widest = 1;
    for (int p = 0; p < 3; ++p) widest = std::max(widest, ptot[p]);
    b->grid = (int)std::min<long long>((long long)std::max(1, per_sm) * sms,
                                       std::max<long long>(sms, widest));
    b->dirty = false;
    return GP_OK;
}

int batch_sync_errors(gp_batch *b)
{
    GP_BCK(b, cudaMemcpyAsync(b->h_err, b->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    GP_BCK(b, cudaStreamSynchronize(b->stream));
    const int bits = b->h_err[0];
    if (bits) {
        // reported once: the next calls start clean
        GP_BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
        GP_BCK(b, cudaStreamSynchronize(b->stream));
    }
    if (bits & 2) return bfail(b, GP_ETIMEOUT, "a batched step's bounded dependency wait gave up");
    if (bits & 1) return bfail(b, GP_ENONFINITE, "a norm became non-finite or zero");
    return GP_OK;
}

int materialize(gp_batch *b, gp_batch_slot &s)
{
    if (!s.scale_pending) return GP_OK;
    const long long n = (long long)s.grid.nx * s.grid.ny * s.grid.nz;
    const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
    if (b->prec == GP_C128) k_batch_apply_scale<double><<<blocks, 256, 0, b->stream>>>((double2 *)s.psi, n, s.scale);
    else k_batch_apply_scale<float><<<blocks, 256, 0, b->stream>>>((float2 *)s.psi, n, s.scale);
    GP_BCK(b, cudaGetLastError());
    k_batch_set_one<<<1, 1, 0, b->stream>>>(s.scale);
    GP_BCK(b, cudaGetLastError());
    s.scale_pending = false;
    return GP_OK;
}

bool valid_slot(gp_batch *b, int slot)
{
    return b && slot >= 0 && slot < (int)b->slots.size() && b->slots[slot].used;
}

// Observables of the active instances b->active[sel[i]] into out[i]
// (prepared batch); synchronises.  Each instance's sums run over its own
// rows in a fixed order, so a result does not depend on the subset.
int observe(gp_batch *b, const std::vector<int> &sel, gp_obs *out)
{
    const int M = (int)sel.size();
    if (M == 0) return GP_OK;
    long long *pref = reinterpret_cast<long long *>(b->h_sub);
    int *idx = reinterpret_cast<int *>(pref + M + 1);
    pref[0] = 0;
    for (int i = 0; i < M; ++i) {
        idx[i] = sel[i];
        const gp_grid &g = b->slots[b->active[sel[i]]].grid;
        pref[i + 1] = pref[i] + obs_groups(g.ny, g.nz);
    }
    const size_t bytes = (M + 1) * sizeof(long long) + M * sizeof(int);
    GP_BCK(b, cudaMemcpyAsync(b->d_sub, b->h_sub, bytes, cudaMemcpyHostToDevice, b->stream));
    const long long *d_pref = reinterpret_cast<const long long *>(b->d_sub);
    const int *d_idx = reinterpret_cast<const int *>(d_pref + M + 1);
    const unsigned blocks = (unsigned)((pref[M] * 32 + 255) / 256);
    if (b->prec == GP_C128) k_batch_obs<double><<<blocks, 256, 0, b->stream>>>(b->d_inst, d_idx, d_pref, M);
    else k_batch_obs<float><<<blocks, 256, 0, b->stream>>>(b->d_inst, d_idx, d_pref, M);
    GP_BCK(b, cudaGetLastError());
    k_batch_obs_finish<<<M, 256, 0, b->stream>>>(b->d_inst, d_idx, b->d_sums);
    GP_BCK(b, cudaGetLastError());
    GP_BCK(b, cudaMemcpyAsync(b->h_sums, b->d_sums, M * gp::kObsWidth * sizeof(double),
                              cudaMemcpyDeviceToHost, b->stream));
    const int rc = batch_sync_errors(b);     // (also makes h_sub reusable)
    int bad = 0;
    for (int i = 0; i < M; ++i) {
        const gp_batch_slot &s = b->slots[b->active[sel[i]]];
        const double *q = b->h_sums + (size_t)i * gp::kObsWidth;
        const double w = s.h[0] * s.h[1] * (s.grid.nz > 1 ? s.h[2] : 1.0);
        const double nrm = w * q[0];
        double kin = 0.5 * (q[6] / (s.h[0] * s.h[0]) + q[7] / (s.h[1] * s.h[1]));
        if (s.grid.nz > 1) kin += 0.5 * q[8] / (s.h[2] * s.h[2]);
        gp_obs &o = out[i];
        std::memset(&o, 0, sizeof(gp_obs));
        o.norm = nrm;
        o.mu = w * (kin + q[4] + s.g * q[5]) / nrm;
        o.energy = w * (kin + q[4] + 0.5 * s.g * q[5]) / nrm;
        o.rms_x = std::sqrt(q[1] / q[0]);
        o.rms_y = std::sqrt(q[2] / q[0]);
        o.rms_z = std::sqrt(q[3] / q[0]);
        o.rms_r = std::sqrt((q[1] + q[2] + q[3]) / q[0]);
        o.step = s.step;
        o.t = s.step * s.dt;
        if (!std::isfinite(o.mu) || !std::isfinite(o.norm)) bad = 1;
    }
    if (rc) return rc;
    if (bad) return bfail(b, GP_ENONFINITE, "gp_batch_observables: non-finite result");
    return GP_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int gp_batch_footprint(const gp_grid *grid, int precision, size_t *bytes)
{
    if ((precision != GP_C128 && precision != GP_C64) || !batch_grid_ok(grid, precision) || !bytes)
        return bfail(nullptr, GP_EINVAL, "gp_batch_footprint: invalid grid or precision");
    *bytes = slot_bytes(*grid, precision);
    return GP_OK;
}

int gp_batch_create(int precision, size_t cap_bytes, void *cuda_stream, gp_batch **out)
{
    if (out) *out = nullptr;
    if (!out || (precision != GP_C128 && precision != GP_C64) || cap_bytes == 0)
        return bfail(nullptr, GP_EINVAL, "gp_batch_create: bad precision or zero cap");
    gp_batch *b = new (std::nothrow) gp_batch;
    if (!b) return bfail(nullptr, GP_ENOMEM, "gp_batch_create: host allocation failed");
    b->prec = precision;
    b->cap = cap_bytes;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_head, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_err, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_err, 2 * sizeof(int));
    if (e != cudaSuccess) {
        std::string msg = std::string("gp_batch_create: ") + cudaGetErrorString(e);
        gp_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA, msg);
    }
    *out = b;
    return GP_OK;
}

int gp_batch_add(gp_batch *b, const gp_grid *grid, const double dx[3], double dt, double gamma,
                 double nu, double lambda, double g, int mode, int *slot)
{
    if (slot) *slot = -1;
    if (!b || !slot || !dx) return bfail(b, GP_EINVAL, "gp_batch_add: null argument");
    if (!batch_grid_ok(grid, b->prec))
        return bfail(b, GP_EINVAL, "gp_batch_add: invalid grid (edges 3 .. 512 complex64, 384 complex128; nz == 1 for 2D)");
    const int nd = grid->nz > 1 ? 3 : 2;
    for (int k = 0; k < nd; ++k)
        if (!(dx[k] > 0) || !std::isfinite(dx[k])) return bfail(b, GP_EINVAL, "gp_batch_add: dx must be > 0");
    if (!(dt > 0) || !std::isfinite(dt) || !(gamma >= 0) || !(nu >= 0) || !(lambda >= 0) ||
        !std::isfinite(g) || (mode != GP_IMAG && mode != GP_REAL))
        return bfail(b, GP_EINVAL, "gp_batch_add: bad dt, trap, g or mode");
    const size_t bytes = slot_bytes(*grid, b->prec);
    if (b->used + bytes > b->cap) return bfail(b, GP_EFULL, "gp_batch_add: the memory cap is reached");
    int id = -1;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (!b->slots[i].used) { id = (int)i; break; }
    if (id < 0) {
        b->slots.emplace_back();
        id = (int)b->slots.size() - 1;
    }
    gp_batch_slot &s = b->slots[id];
    s = gp_batch_slot{};
    s.grid = *grid;
    s.h[0] = dx[0];
    s.h[1] = dx[1];
    s.h[2] = nd == 3 ? dx[2] : 1.0;
    s.dt = dt;
    s.w[0] = gamma;
    s.w[1] = nu;
    s.w[2] = nd == 3 ? lambda : 0.0;
    s.g = g;
    s.mode = mode;
    s.bytes = bytes;
    const size_t psi_bytes = (size_t)grid->nx * grid->ny * grid->nz * elem(b->prec);
    cudaError_t e = cudaMallocAsync(&s.psi, psi_bytes, b->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&s.aux, aux_layout(s.grid, b->prec).total, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.psi, 0, psi_bytes, b->stream);
    if (e != cudaSuccess) {
        if (s.psi) cudaFreeAsync(s.psi, b->stream);
        if (s.aux) cudaFreeAsync(s.aux, b->stream);
        s = gp_batch_slot{};
        return bfail(b, e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA,
                     std::string("gp_batch_add: ") + cudaGetErrorString(e));
    }
    s.used = true;
    int rc = upload_slot(b, s);
    if (rc) {
        cudaFreeAsync(s.psi, b->stream);
        cudaFreeAsync(s.aux, b->stream);
        s = gp_batch_slot{};
        return rc;
    }
    b->used += bytes;
    b->dirty = true;
    *slot = id;
    return GP_OK;
}

int gp_batch_load(gp_batch *b, int slot, const void *psi, int64_t count, int on_device)
{
    if (!valid_slot(b, slot)) return bfail(b, GP_EINVAL, "gp_batch_load: bad slot");
    gp_batch_slot &s = b->slots[slot];
    const long long n = (long long)s.grid.nx * s.grid.ny * s.grid.nz;
    s.step = 0;
    s.scale_pending = false;
    if (!psi) {
        GP_BCK(b, gp::launch_seed(b->prec, s.psi, s.grid.nx, s.grid.ny, s.grid.nz, s.h, s.w, b->stream));
        // normalise: FP64 norm partials over the seed, finish into the scale
        double *part = s.obs_rows;          // scratch: the rows are rewritten by observables
        gp::Partials pp{part, 1};
        const int blocks = (int)std::min<long long>(lines_of(s.grid, 0) * gp::kObsWidth, gp::kReduceBlocks);
        GP_BCK(b, gp::launch_norm_partials(b->prec, s.psi, n, pp, blocks, b->stream));
        const double w = s.h[0] * s.h[1] * (s.grid.nz > 1 ? s.h[2] : 1.0);
        GP_BCK(b, gp::launch_norm_finish(part, blocks, w, s.scale, s.norm, b->d_err, b->stream));
        s.scale_pending = true;
        int rc = materialize(b, s);
        if (rc) return rc;
        GP_BCK(b, cudaStreamSynchronize(b->stream));
        return GP_OK;
    }
    if (count != n) return bfail(b, GP_EINVAL, "gp_batch_load: count != nx*ny*nz");
    GP_BCK(b, cudaMemcpyAsync(s.psi, psi, (size_t)n * elem(b->prec),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
    GP_BCK(b, gp::launch_zero_boundary(b->prec, s.psi, s.grid.nx, s.grid.ny, s.grid.nz, b->stream));
    k_batch_set_one<<<1, 1, 0, b->stream>>>(s.scale);
    GP_BCK(b, cudaGetLastError());
    GP_BCK(b, cudaStreamSynchronize(b->stream));
    return GP_OK;
}

int gp_batch_store(gp_batch *b, int slot, void *out, int64_t count, int on_device)
{
    if (!valid_slot(b, slot) || !out) return bfail(b, GP_EINVAL, "gp_batch_store: bad slot or buffer");
    gp_batch_slot &s = b->slots[slot];
    const long long n = (long long)s.grid.nx * s.grid.ny * s.grid.nz;
    if (count != n) return bfail(b, GP_EINVAL, "gp_batch_store: count != nx*ny*nz");
    int rc = materialize(b, s);
    if (rc) return rc;
    GP_BCK(b, cudaMemcpyAsync(out, s.psi, (size_t)n * elem(b->prec),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    GP_BCK(b, cudaStreamSynchronize(b->stream));
    return batch_sync_errors(b);
}

int gp_batch_set_params(gp_batch *b, int slot, double g, int mode)
{
    if (!valid_slot(b, slot) || !std::isfinite(g) || (mode != GP_IMAG && mode != GP_REAL))
        return bfail(b, GP_EINVAL, "gp_batch_set_params: bad slot, g or mode");
    gp_batch_slot &s = b->slots[slot];
    if (mode != s.mode) {
        int rc = materialize(b, s);
        if (rc) return rc;
    }
    s.g = g;
    s.mode = mode;
    b->dirty = true;
    return GP_OK;
}

int gp_batch_remove(gp_batch *b, int slot)
{
    if (!valid_slot(b, slot)) return bfail(b, GP_EINVAL, "gp_batch_remove: bad slot");
    gp_batch_slot &s = b->slots[slot];
    cudaFreeAsync(s.psi, b->stream);
    cudaFreeAsync(s.aux, b->stream);
    b->used -= s.bytes;
    s = gp_batch_slot{};
    b->dirty = true;
    return GP_OK;
}

int gp_batch_set_wait_ns(gp_batch *b, int64_t ns)
{
    if (!b || ns < 0) return bfail(b, GP_EINVAL, "gp_batch_set_wait_ns: need ns >= 0");
    b->wait_ns = (unsigned long long)ns;
    return GP_OK;
}

int gp_batch_step(gp_batch *b, int64_t n)
{
    if (!b || n < 0) return bfail(b, GP_EINVAL, "gp_batch_step: bad arguments");
    int rc = prepare(b);
    if (rc) return rc;
    if (n == 0 || b->active.empty()) return GP_OK;
    LaunchArgs A = b->args;
    A.wait_ns = b->wait_ns;
    const int N = A.N;
    // at most 2^31 items per launch: split long runs into chunks of steps
    const long long max_steps = std::max<long long>(1, (1LL << 30) / std::max<long long>(1, A.ips));
    for (int64_t done = 0; done < n;) {
        const int k = (int)std::min<long long>(n - done, max_steps);
        A.steps = k;
        GP_BCK(b, cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), b->stream));
        GP_BCK(b, cudaMemsetAsync(A.done, 0, N * sizeof(int), b->stream));
        GP_BCK(b, cudaMemsetAsync(A.abort_flag, 0, sizeof(int), b->stream));
        if (b->prec == GP_C128) k_batch_steps<double><<<b->grid, 32, b->smem, b->stream>>>(A);
        else k_batch_steps<float><<<b->grid, 32, b->smem, b->stream>>>(A);
        GP_BCK(b, cudaGetLastError());
        done += k;
    }
    for (int id : b->active) {
        b->slots[id].step += n;
        if (b->slots[id].mode == GP_IMAG) b->slots[id].scale_pending = true;
    }
    return GP_OK;
}

int gp_batch_observables(gp_batch *b, gp_obs *out, int capacity)
{
    if (!b || (!out && capacity > 0)) return bfail(b, GP_EINVAL, "gp_batch_observables: null argument");
    int rc = prepare(b);
    if (rc) return rc;
    for (int i = 0; i < capacity; ++i) {
        std::memset(&out[i], 0, sizeof(gp_obs));
        out[i].step = -1;
    }
    const int N = (int)b->active.size();
    std::vector<int> all(N);
    for (int a = 0; a < N; ++a) all[a] = a;
    std::vector<gp_obs> got(N);
    rc = observe(b, all, got.data());
    for (int a = 0; a < N; ++a)
        if (b->active[a] < capacity) out[b->active[a]] = got[a];
    return rc;
}

int gp_batch_observables_of(gp_batch *b, const int *slots, int count, gp_obs *out)
{
    if (!b || count < 0 || (count > 0 && (!slots || !out)))
        return bfail(b, GP_EINVAL, "gp_batch_observables_of: null argument or count < 0");
    for (int i = 0; i < count; ++i)
        if (!valid_slot(b, slots[i])) return bfail(b, GP_EINVAL, "gp_batch_observables_of: bad slot");
    int rc = prepare(b);
    if (rc) return rc;
    std::vector<int> pos(b->slots.size(), -1), sel(count);
    for (size_t a = 0; a < b->active.size(); ++a) pos[b->active[a]] = (int)a;
    for (int i = 0; i < count; ++i) sel[i] = pos[slots[i]];
    return observe(b, sel, out);
}

int gp_batch_info(gp_batch *b, int *active, int *slots, size_t *used_bytes)
{
    if (!b) return bfail(nullptr, GP_EINVAL, "gp_batch_info: null batch");
    int n = 0;
    for (const auto &s : b->slots) n += s.used ? 1 : 0;
    if (active) *active = n;
    if (slots) *slots = (int)b->slots.size();
    if (used_bytes) *used_bytes = b->used;
    return GP_OK;
}

int gp_batch_sync(gp_batch *b)
{
    if (!b) return bfail(nullptr, GP_EINVAL, "gp_batch_sync: null batch");
    GP_BCK(b, cudaStreamSynchronize(b->stream));
    return batch_sync_errors(b);
}

const char *gp_batch_last_error(const gp_batch *b)
{
    return b ? b->last_error.c_str() : gp_last_error(nullptr);
}

void gp_batch_destroy(gp_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &s : b->slots) {
        if (s.psi) cudaFreeAsync(s.psi, b->stream);
        if (s.aux) cudaFreeAsync(s.aux, b->stream);
    }
    if (b->d_inst) cudaFreeAsync(b->d_inst, b->stream);
    if (b->d_ints) cudaFreeAsync(b->d_ints, b->stream);
    if (b->d_sub) cudaFreeAsync(b->d_sub, b->stream);
    if (b->d_sums) cudaFreeAsync(b->d_sums, b->stream);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->d_head) cudaFree(b->d_head);
    if (b->d_err) cudaFree(b->d_err);
    if (b->h_sums) cudaFreeHost(b->h_sums);
    if (b->h_sub) cudaFreeHost(b->h_sub);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
