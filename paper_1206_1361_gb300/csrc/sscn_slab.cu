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
    // rows to warps, points of a row to lanes (coalesced, no index division)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int y = warp; y < ny; y += nwarps)
        for (int x = lane; x < nx; x += 32) cp_async<(int)sizeof(C)>(&sm[y * P + x], &plane[y * nx + x]);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int r = warp * 16 + (lane & 15);                 // this lane pair's line
    const bool top = lane < 16;
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
    __syncthreads();
    for (int y = warp; y < ny; y += nwarps)
        for (int x = lane; x < nx; x += 32) plane[y * nx + x] = sm[y * P + x];
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

}  // namespace

size_t slab_bytes(int prec, int nx, int ny)
{
    return (size_t)ny * (size_t)(nx | 1) * (prec == kC128 ? 16 : 8);
}

bool slab_fits(int prec, int nx, int ny)
{
    return nx >= 3 && ny >= 3 && nx <= kMaxSlabEdge && ny <= kMaxSlabEdge &&
           slab_bytes(prec, nx, ny) <= (size_t)kMaxSlabBytes;
}

cudaError_t launch_sweep_xy(int prec, int mode, void *psi, int nx, int ny, int nz,
                            const AxisTables &ax, const AxisTables &ay, const NonlinArgs &nl,
                            cudaStream_t st)
{
    if (!slab_fits(prec, nx, ny) || nz < 1) return cudaErrorInvalidValue;
    if (prec == kC128)
        return mode == 0 ? launch_xy<double, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                         : launch_xy<double, 1>(psi, nx, ny, nz, ax, ay, nl, st);
    return mode == 0 ? launch_xy<float, 0>(psi, nx, ny, nz, ax, ay, nl, st)
                     : launch_xy<float, 1>(psi, nx, ny, nz, ax, ay, nl, st);
}

}  // namespace gp
