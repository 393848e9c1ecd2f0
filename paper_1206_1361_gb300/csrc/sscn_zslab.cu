// sscn_zslab.cu -- kernels of the z-slab decomposition of one grid over
// several GPUs (FP64, real time).
//
// Rank r holds the z-planes [b_r, b_{r+1}) of the grid (rank 0 from the
// Dirichlet plane 0) as an ordinary context whose first local plane is a zero
// plane (for r > 0 a stand-in for the neighbour's last plane), so the x and y
// sweeps and calcnu run unchanged, and the context's z sweep solves its block
// A_r v_r = psi_r of the z lines with zero coupling at both ends (A = I -
// kappa L).  The coupling is restored afterwards (the partitioned, "spike"
// form of the tridiagonal solve): with s_r = A_r^{-1} (kappa e_first) and
// t_r = A_r^{-1} (kappa e_last),
//     v_r = y_r + s_r L_{r-1} + t_r F_{r+1},   y_r = A_r^{-1} psi_r,
// where F_q, L_q are the solution's values on rank q's first and last unknown
// planes.  Those satisfy, line by line, the reduced system
//     F_q = yF_q + sF_q L_{q-1} + tF_q F_{q+1},   L_q = yL_q + sL_q L_{q-1} + tL_q F_{q+1}
// (L_{-1} = F_P = 0) in the 2 (P - 1) unknowns L_0 .. L_{P-2}, F_1 .. F_{P-1};
// the ranks exchange their yF, yL planes (an all-gather); the reduced matrix
// is the same on every line, so each rank holds the two rows of its inverse
// that give L_{r-1} and F_{r+1} and corrects its planes,
//     u_r = u_loc + 2 (s_r L_{r-1} + t_r F_{r+1}),
// u_loc = 2 y_r - psi_r being what the local z sweep wrote.

#include <cuda_runtime.h>

#include "sscn_internal.h"

namespace gp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double coordg(int n, double h, int i) { return -0.5 * n * h + i * h; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_slab_seed(double2 *__restrict__ psi, int nx, int ny, int nzl, int nzg, int z0,
                            double hx, double hy, double hz, double gx, double gy, double gz)
{
    const long long count = (long long)nx * ny * nzl;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % nx);
        const int j = (int)((p / nx) % ny);
        const int k = (int)(p / ((long long)nx * ny));
        double v = 0.0;
        if (i > 0 && j > 0 && k > 0) {
            const double x = coordg(nx, hx, i), y = coordg(ny, hy, j), z = coordg(nzg, hz, z0 + k);
            v = exp(-0.5 * (gx * x * x + gy * y * y + gz * z * z));
        }
        psi[p] = make_double2(v, 0.0);
    }
}

// saved[0 .. plane) <- psi at local plane kf, saved[plane .. 2 plane) <- at kl
__global__ void k_slab_capture(const double2 *__restrict__ psi, double2 *__restrict__ saved,
                               long long plane, int kf, int kl)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < plane;
         p += (long long)gridDim.x * blockDim.x) {
        saved[p] = psi[kf * plane + p];
        saved[plane + p] = psi[kl * plane + p];
    }
}

// y = (u_loc + psi) / 2 on the first and last unknown planes
__global__ void k_slab_bnd(const double2 *__restrict__ psi, const double2 *__restrict__ saved,
                           double2 *__restrict__ bnd, long long plane, int kf, int kl)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < plane;
         p += (long long)gridDim.x * blockDim.x) {
        const double2 a = psi[kf * plane + p], b = saved[p];
        const double2 c = psi[kl * plane + p], d = saved[plane + p];
        bnd[p] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
        bnd[plane + p] = make_double2(0.5 * (c.x + d.x), 0.5 * (c.y + d.y));
    }
}

// Per z line: alpha = L_{r-1} and beta = F_{r+1} of the reduced system's
// solution as the linear combinations w of the gathered boundary values (the
// reduced matrix is the same on every line, so the host inverts it once and
// hands over the two rows this rank needs), then the correction of the
// rank's unknown planes 1 .. nloc.  w[(2 q + e)] (alpha) and w[2 P + 2 q + e]
// (beta) weigh rank q's first (e = 0) and last (e = 1) boundary plane.
__global__ void __launch_bounds__(kThreads)
k_slab_correct(double2 *__restrict__ psi, const double2 *__restrict__ bnd_all,
               const double2 *__restrict__ w, const double2 *__restrict__ spike, int P,
               long long plane, int nloc)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= plane) return;
    double2 al = make_double2(0.0, 0.0), be = make_double2(0.0, 0.0);
    for (int j = 0; j < 2 * P; ++j) {
        const double2 y = bnd_all[(long long)j * plane + p];
        const double2 a = cmul(w[j], y), b = cmul(w[2 * P + j], y);
        al = make_double2(al.x + a.x, al.y + a.y);
        be = make_double2(be.x + b.x, be.y + b.y);
    }
    for (int k = 1; k <= nloc; ++k) {
        const double2 s = spike[k - 1], t = spike[nloc + k - 1];
        const double2 c1 = cmul(s, al), c2 = cmul(t, be);
        double2 &u = psi[k * plane + p];
        u = make_double2(u.x + 2.0 * (c1.x + c2.x), u.y + 2.0 * (c1.y + c2.y));
    }
}

// partials[b] = sum over this block's lines of Re(next * conj(last))
__global__ void __launch_bounds__(kThreads)
k_slab_interface(const double2 *__restrict__ last, const double2 *__restrict__ next, long long plane,
                 double *__restrict__ partials)
{
    __shared__ double red[kThreads / 32];
    double v = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < plane;
         p += (long long)gridDim.x * blockDim.x)
        v += next[p].x * last[p].x + next[p].y * last[p].y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_slab_sum(const double *__restrict__ partials, int count, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < count; ++b) s += partials[b];
        *out = s;
    }
}

int blocks_for(long long n)
{
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > kReduceBlocks ? kReduceBlocks : b));
}

}  // namespace

cudaError_t launch_slab_seed(void *psi, int nx, int ny, int nzl, int nzg, int z0, const double h[3],
                             const double w[3], cudaStream_t st)
{
    k_slab_seed<<<blocks_for((long long)nx * ny * nzl), kThreads, 0, st>>>(
        (double2 *)psi, nx, ny, nzl, nzg, z0, h[0], h[1], h[2], w[0], w[1], w[2]);
    return cudaGetLastError();
}

cudaError_t launch_slab_capture(const void *psi, void *saved, long long plane, int kf, int kl,
                                cudaStream_t st)
{
    k_slab_capture<<<blocks_for(plane), kThreads, 0, st>>>((const double2 *)psi, (double2 *)saved,
                                                           plane, kf, kl);
    return cudaGetLastError();
}

cudaError_t launch_slab_bnd(const void *psi, const void *saved, void *bnd, long long plane, int kf,
                            int kl, cudaStream_t st)
{
    k_slab_bnd<<<blocks_for(plane), kThreads, 0, st>>>((const double2 *)psi, (const double2 *)saved,
                                                       (double2 *)bnd, plane, kf, kl);
    return cudaGetLastError();
}

cudaError_t launch_slab_correct(void *psi, const void *bnd_all, const double2 *w,
                                const double2 *spike, int P, long long plane, int nloc,
                                cudaStream_t st)
{
    if (P < 1 || P > kSlabMaxRanks) return cudaErrorInvalidValue;
    if (P == 1) return cudaSuccess;
    const long long blocks = (plane + kThreads - 1) / kThreads;
    k_slab_correct<<<(unsigned)blocks, kThreads, 0, st>>>((double2 *)psi, (const double2 *)bnd_all,
                                                          w, spike, P, plane, nloc);
    return cudaGetLastError();
}

cudaError_t launch_slab_interface(const void *last_plane, const void *next_plane, long long plane,
                                  double *partials, double *out, cudaStream_t st)
{
    const int blocks = blocks_for(plane);
    k_slab_interface<<<blocks, kThreads, 0, st>>>((const double2 *)last_plane,
                                                  (const double2 *)next_plane, plane, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_slab_sum<<<1, 32, 0, st>>>(partials, blocks, out);
    return cudaGetLastError();
}

}  // namespace gp
