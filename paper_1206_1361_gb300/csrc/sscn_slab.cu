// sscn_slab.cu -- the x and y Crank-Nicolson sweeps (calclux, calcluy) of
// one step fused into a single pass over the grid: one CTA holds a whole
// z-plane in shared memory, runs calcnu with the x sweep on its rows and the
// y sweep on its columns there, and writes the plane back.  psi then moves
// through HBM twice per step (this pass and the z sweep) instead of three
// times: 32 (complex128) / 16 (complex64) bytes per point and step saved.
//
// Plane layout in shared memory: row y at y P, P = nx | 1 (odd pitch), so a
// warp's 16 rows read at one column, and its 16 columns read at one row,
// fall in distinct banks.  Each line is solved in place by a lane pair
// (gp::solve_pair, right-hand-side form, two-ended), 16 lines per warp; the
// same CTA does the rows, then (after a barrier) the columns.
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "sscn_pair.cuh"
#include "sscn_slab.h"

namespace gp {
namespace {

constexpr int kMaxSlabBytes = 232448;      // opt-in shared memory of one CTA
constexpr int kMaxSlabEdge = 256;          // 2 lanes per line, 512 threads

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int BYTES> __device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <typename T> PairTabs<T> pair_tabs(const AxisTables &a, int mode)
{
    PairTabs<T> t;
    const double kap = mode == 0 ? a.kre : a.kim;
    t.kappa = (T)kap;
    if constexpr (sizeof(T) == 8) {
        t.mult = a.mult64;
        t.cp = a.cp64;
        t.minf = a.minf64;
        t.cinf = a.cinf64;
        t.mid = a.mid64;
        t.conv = a.conv64;
    } else {
        t.mult = a.mult32;
        t.cp = a.cp32;
        t.minf = a.minf32;
        t.cinf = a.cinf32;
        t.mid = a.mid32;
        t.conv = a.conv32;
    }
    return t;
}

// One CTA per z-plane (blockIdx.x = k); 32 ceil(max(nx, ny) / 16) threads.
// Calcnu tables in x, y, z order (px along the rows, py[j], pz[k]).
template <typename T, int MODE>
__global__ void __launch_bounds__(512)
k_sweep_xy(typename Cx<T>::t *__restrict__ psi, int nx, int ny, PairTabs<T> tx, PairTabs<T> ty,
           const typename Coef<T>::t *px, const typename Coef<T>::t *py,
           const typename Coef<T>::t *pz, const float *thx, const float *thy, const float *thz,
           StepG sg, const double *scale)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char slab_raw[];
    C *sm = reinterpret_cast<C *>(slab_raw);
    const int P = nx | 1;
    const int kz = blockIdx.x;
    C *plane = psi + (long long)kz * nx * ny;
    // Each warp loads the 16 rows it sweeps along x and starts on them as soon
    // as its own copies land; one CTA barrier before the columns; each warp
    // then stores the 16 columns it swept along y.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = warp * 16 + (lane & 15);                 // this lane pair's line
    const bool top = lane < 16;
    for (int y = warp * 16; y < min(warp * 16 + 16, ny); ++y)
        for (int x = lane; x < nx; x += 32) cp_async<(int)sizeof(C)>(&sm[y * P + x], &plane[y * nx + x]);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    Acc<T> acc;                                            // (no norm here)
    {
        // x sweep on row r (calcnu fused into its elimination)
        const bool active = r < ny;
        Calcnu<T, MODE> cu{};
        if (active) cu.setup(px, py, pz, thx, thy, thz, r, kz, sg.value(), scale);
        solve_pair<T, MODE, true, 1>(sm + r * P, 1, nx, top, active, false, acc, tx, cu);
    }
    __syncthreads();
    {
        // y sweep on column r
        const bool active = r < nx;
        const Calcnu<T, MODE> none{};
        solve_pair<T, MODE, false, 0>(sm + r, P, ny, top, active, false, acc, ty, none);
    }
    __syncwarp();
    if (r < nx)                                            // lanes 0-15 even rows, 16-31 odd
        for (int y = lane >> 4; y < ny; y += 2) plane[y * nx + r] = sm[y * P + r];
}

// ---- one plane over a 2-CTA cluster ---------------------------------------
// A plane larger than one CTA's shared memory is split across a cluster of
// two CTAs:
// the y lines' two-ended elimination already splits them at the middle row
// k = ceil(m / 2), so CTA 0 holds rows 0 .. k and CTA 1 rows k+1 .. ny-1,
// each with the other's boundary row as a halo (through distributed shared
// memory), and only the values the lane pair of the one-CTA kernel
// exchanges by shuffles cross between the CTAs: e_{k+1} one way, v_k the
// other.  The arithmetic is that of gp::solve_pair, step for step.

// Forward elimination of one half line from its first point p (element
// stride dir, +es top / -es bottom) over len points; the point after the
// last is read (the middle row, or the halo).
template <typename T, int MODE>
__device__ __forceinline__ void half_forward(typename Cx<T>::t *p, int dir, int len,
                                             const PairTabs<T> &tb, const LineOps<T, MODE> &cn,
                                             typename Cx<T>::t &prev, typename Cx<T>::t &cur,
                                             typename Cx<T>::t &d)
{
    using C = typename Cx<T>::t;
    const int tc = min(tb.conv, len);
    cur = *p;
    int t = 0;
    for (; t < tc; ++t, p += dir) {
        const C next = p[dir];
        d = cn.fwd(cn.rhs(prev, cur, next), d, tb.mult[t]);
        *p = d;
        prev = cur;
        cur = next;
    }
    for (; t + 4 <= len; t += 4, p += 4 * dir) {
        C nx[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) nx[q] = p[(q + 1) * dir];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            d = cn.fwd(cn.rhs(prev, cur, nx[q]), d, tb.minf);
            p[q * dir] = d;
            prev = cur;
            cur = nx[q];
        }
    }
    for (; t < len; ++t, p += dir) {
        const C next = p[dir];
        d = cn.fwd(cn.rhs(prev, cur, next), d, tb.minf);
        *p = d;
        prev = cur;
        cur = next;
    }
}

// Back substitution of the same half line from u (the middle row's value),
// points len-1 .. 0 after first.
template <typename T, int MODE>
__device__ __forceinline__ void half_back(typename Cx<T>::t *first, int dir, int len,
                                          const PairTabs<T> &tb, const LineOps<T, MODE> &cn,
                                          typename Cx<T>::t u)
{
    using C = typename Cx<T>::t;
    const int tc = min(tb.conv, len);
    int t = len - 1;
    C *p = first + t * dir;
    for (; t - 3 >= tc; t -= 4, p -= 4 * dir) {
        C dv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dv[q] = p[-q * dir];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            u = cn.back(dv[q], tb.cinf, u);
            p[-q * dir] = u;
        }
    }
    for (; t >= tc; --t, p -= dir) {
        u = cn.back(*p, tb.cinf, u);
        *p = u;
    }
    for (; t >= 0; --t, p -= dir) {
        u = cn.back(*p, tb.cp[t], u);
        *p = u;
    }
}

// Rows per CTA of the split plane (the larger half plus its halo row).
__host__ __device__ __forceinline__ int split_rows(int ny) { return (ny + 1) / 2 + 1 + 1; }

// blockIdx.x = 2 kz + rank.  Shared memory: split_rows(ny) rows of pitch
// nx | 1, then two exchange rows of nx points.  CTA 0: local row = global
// row (halo k+1); CTA 1: local row = global row - k (halo k at 0).
template <typename T, int MODE>
__global__ void __launch_bounds__(512)
k_sweep_xy2(typename Cx<T>::t *__restrict__ psi, int nx, int ny, PairTabs<T> tx, PairTabs<T> ty,
            const typename Coef<T>::t *px, const typename Coef<T>::t *py,
            const typename Coef<T>::t *pz, const float *thx, const float *thy, const float *thz,
            StepG sg, const double *scale)
{
    using C = typename Cx<T>::t;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char slab_raw[];
    C *sm = reinterpret_cast<C *>(slab_raw);
    const int P = nx | 1;
    const int R = split_rows(ny);
    C *xd = sm + R * P, *xv = xd + nx;       // exchange rows (received values)
    const int rank = (int)cl.block_rank();
    const int kz = blockIdx.x >> 1;
    const int m = ny - 1, k = (m + 1) >> 1;
    const int g0 = rank == 0 ? 0 : k + 1;     // first own row
    const int g1 = rank == 0 ? k : m;         // last own row
    const int base = rank == 0 ? 0 : k;       // global row of local row 0
    C *plane = psi + (long long)kz * nx * ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int y = g0 + warp; y <= g1; y += nwarps)
        for (int x = lane; x < nx; x += 32)
            cp_async<(int)sizeof(C)>(&sm[(y - base) * P + x], &plane[y * nx + x]);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    {
        // x sweep on the own rows (lane pairs, calcnu fused)
        const int r = warp * 16 + (lane & 15);
        const int y = g0 + r;
        const bool active = y <= g1;
        Calcnu<T, MODE> cu{};
        if (active) cu.setup(px, py, pz, thx, thy, thz, y, kz, sg.value(), scale);
        Acc<T> acc;
        solve_pair<T, MODE, true, 1>(sm + (active ? y - base : 0) * P, 1, nx, lane < 16, active,
                                     false, acc, tx, cu);
    }
    cl.sync();                                // both halves through the x sweep
    {
        // halo: CTA 0 sends row k, CTA 1 sends row k+1
        C *peer = cl.map_shared_rank(sm, rank ^ 1);
        const int send = rank == 0 ? k : k + 1;
        const int dst = rank == 0 ? 0 : k + 1;   // its local row in the peer
        for (int x = threadIdx.x; x < nx; x += blockDim.x) peer[dst * P + x] = sm[(send - base) * P + x];
    }
    cl.sync();
    const LineOps<T, MODE> cn{ty.kappa};
    const int x = threadIdx.x;
    const bool col = x < nx;
    const C zero = cx<T>((T)0, (T)0);
    C prev = zero, cur = zero, d = zero;
    const int len = rank == 0 ? k - 1 : m - k;
    const int dir = rank == 0 ? P : -P;
    C *first = sm + ((rank == 0 ? 1 : m) - base) * P + x;
    if (col) half_forward<T, MODE>(first, dir, len, ty, cn, prev, cur, d);
    if (rank == 1 && col) cl.map_shared_rank(xd, 0)[x] = d;       // e_{k+1}
    cl.sync();
    C u = zero;
    if (rank == 0 && col) {
        const C o_prev = sm[(k + 1) * P + x];                      // psi_{k+1} (halo)
        const C o_d = xd[x];
        u = cn.fwd(cn.rhs(prev, cur, o_prev), cx<T>(d.x + o_d.x, d.y + o_d.y), ty.mid);
        sm[k * P + x] = u;
        cl.map_shared_rank(xv, 1)[x] = u;                           // v_k
    }
    cl.sync();
    if (rank == 1 && col) u = xv[x];
    if (col) half_back<T, MODE>(first, dir, len, ty, cn, u);
    __syncthreads();
    for (int y = g0 + warp; y <= g1; y += nwarps)
        for (int x2 = lane; x2 < nx; x2 += 32) plane[y * nx + x2] = sm[(y - base) * P + x2];
}

template <typename T, int MODE>
cudaError_t launch_xy(void *psi, int nx, int ny, int nz, const AxisTables &ax,
                      const AxisTables &ay, const NonlinArgs &nl, cudaStream_t st)
{
    using F = typename Coef<T>::t;
    auto kern = k_sweep_xy<T, MODE>;
    static bool configured[64] = {};          // per device ordinal
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSlabBytes);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const F *px, *py, *pz;
    if constexpr (sizeof(T) == 8) {
        px = nl.px;
        py = nl.py;
        pz = nl.pz;
    } else {
        px = nl.px32;
        py = nl.py32;
        pz = nl.pz32;
    }
    const int threads = 32 * ((std::max(nx, ny) + 15) / 16);
    const size_t smem = slab_bytes(sizeof(T) == 8 ? kC128 : kC64, nx, ny);
    kern<<<nz, threads, smem, st>>>(static_cast<typename Cx<T>::t *>(psi), nx, ny,
                                    pair_tabs<T>(ax, MODE), pair_tabs<T>(ay, MODE), px, py, pz,
                                    nl.tx32, nl.ty32, nl.tz32, nl.g, nl.scale);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_xy2(void *psi, int nx, int ny, int nz, const AxisTables &ax,
                       const AxisTables &ay, const NonlinArgs &nl, cudaStream_t st)
{
    using F = typename Coef<T>::t;
    auto kern = k_sweep_xy2<T, MODE>;
    static bool configured[64] = {};          // per device ordinal
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSlabBytes);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const F *px, *py, *pz;
    if constexpr (sizeof(T) == 8) {
        px = nl.px;
        py = nl.py;
        pz = nl.pz;
    } else {
        px = nl.px32;
        py = nl.py32;
        pz = nl.pz32;
    }
    const int own = (ny - 1 + 1) / 2 + 1;     // rows of CTA 0 (the larger half)
    const int warps = std::max((own + 15) / 16, (nx + 31) / 32);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * nz);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = split_bytes(sizeof(T) == 8 ? kC128 : kC64, nx, ny);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, static_cast<typename Cx<T>::t *>(psi), nx, ny,
                           pair_tabs<T>(ax, MODE), pair_tabs<T>(ay, MODE), px, py, pz, nl.tx32,
                           nl.ty32, nl.tz32, nl.g, nl.scale);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

size_t slab_bytes(int prec, int nx, int ny)
{
    return (size_t)ny * (size_t)(nx | 1) * (prec == kC128 ? 16 : 8);
}

size_t split_bytes(int prec, int nx, int ny)
{
    return ((size_t)split_rows(ny) * (size_t)(nx | 1) + 2 * (size_t)nx) * (prec == kC128 ? 16 : 8);
}

// Over a 2-CTA cluster only when one CTA cannot hold the plane: measured on
// a 128 x 128 complex64 grid, three half-plane CTAs per SM ran no faster than
// one whole-plane CTA (the four cluster barriers per plane eat the overlap),
// and in FP64 the split is slower.
bool slab_split(int prec, int nx, int ny)
{
    return slab_bytes(prec, nx, ny) > (size_t)kMaxSlabBytes;
}

bool slab_fits(int prec, int nx, int ny)
{
    if (nx < 3 || ny < 3 || nx > kMaxSlabEdge || ny > kMaxSlabEdge) return false;
    return slab_split(prec, nx, ny) ? split_bytes(prec, nx, ny) <= (size_t)kMaxSlabBytes
                                    : slab_bytes(prec, nx, ny) <= (size_t)kMaxSlabBytes;
}

cudaError_t launch_sweep_xy(int prec, int mode, void *psi, int nx, int ny, int nz,
                            const AxisTables &ax, const AxisTables &ay, const NonlinArgs &nl,
                            cudaStream_t st)
{
    if (!slab_fits(prec, nx, ny) || nz < 1) return cudaErrorInvalidValue;
    if (slab_split(prec, nx, ny)) {
        if (prec == kC128)
            return mode == 0 ? launch_xy2<double, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                             : launch_xy2<double, 1>(psi, nx, ny, nz, ax, ay, nl, st);
        return mode == 0 ? launch_xy2<float, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                         : launch_xy2<float, 1>(psi, nx, ny, nz, ax, ay, nl, st);
    }
    if (prec == kC128)
        return mode == 0 ? launch_xy<double, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                         : launch_xy<double, 1>(psi, nx, ny, nz, ax, ay, nl, st);
    return mode == 0 ? launch_xy<float, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                     : launch_xy<float, 1>(psi, nx, ny, nz, ax, ay, nl, st);
}

}  // namespace gp
