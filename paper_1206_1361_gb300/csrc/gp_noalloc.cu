// gp_noalloc.cu -- one Crank-Nicolson sweep on a caller-owned device psi,
// without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's operator and may only touch the buffers it was handed (their
// device memory belongs to that framework's allocator), and latency-bound
// loops that must not take cudaMalloc / cudaFree's implicit device-wide
// synchronisation.  For them the sweep's forward-elimination scratch (d'_i,
// one complex value per grid point) and its coefficient tables live in the
// file-scope device array below instead of context-owned memory.  Every GPU
// that loads libgp holds this array (16 MiB plus 512 KiB of tables) until the
// process exits.

#include <cmath>
#include <complex>
#include <vector>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/gp.h"
#include "sscn_internal.h"

namespace {

// Largest grid the static scratch serves: 2^20 complex128 (16 B) points, or
// 2^21 complex64 points.
constexpr size_t kScratchBytes = size_t(1) << 24;
constexpr size_t kTableEntries = GP_MAX_EDGE;
constexpr size_t kTableBytes = kTableEntries * (2 * sizeof(double2) + 2 * sizeof(float4));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes + kTableBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;                       // guards the fields below
void *g_scratch_addr[kMaxDevices];        // device address per device ordinal
// host working arrays of the table recurrence (its constant tails and
// derived fields are passed to the kernels by value)
double2 g_cp64[kTableEntries], g_mult64[kTableEntries];
float4 g_cp32[kTableEntries], g_mult32[kTableEntries];

int reject(int code, const char *msg)
{
    gp::set_thread_error(msg);
    return code;
}

__device__ float4 split_rn(double2 v)
{
    const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
    return make_float4(hx, hy, __double2float_rn(__dsub_rn(v.x, (double)hx)),
                       __double2float_rn(__dsub_rn(v.y, (double)hy)));
}

// The sweep's Thomas tables, written on the device into the table part of the
// static array (nothing is staged through host memory, so the call does not
// wait for earlier work on the stream).  Thread 0 runs the FP64 recurrence up
// to conv64, the index from which the host (running the same explicitly
// rounded recurrence) found every entry equal to the last; thread 32 runs
// the recurrence of the FP32-rounded kappa for the complex64 tables (hi + lo
// pairs) up to conv32; then all threads fill the constant tails.
__global__ void k_noalloc_tables(int m, int conv64, int conv32, double kre, double kim,
                                 double kre32, double kim32, double2 *cp64, double2 *mult64,
                                 float4 *cp32, float4 *mult32)
{
    __shared__ double2 tail[4];
    if (threadIdx.x == 0 || threadIdx.x == 32) {
        const bool f64 = threadIdx.x == 0;
        const double kr = f64 ? kre : kre32, ki = f64 ? kim : kim32;
        const int last = f64 ? conv64 : conv32;
        double2 prev = make_double2(0.0, 0.0), mu = prev, c = prev;
        for (int i = 0; i <= last; ++i) {
            gp::thomas_step(kr, ki, prev.x, prev.y, mu, c);
            if (f64) {
                cp64[i] = c;
                mult64[i] = mu;
            } else {
                cp32[i] = split_rn(c);
                mult32[i] = split_rn(mu);
            }
            prev = c;
        }
        tail[f64 ? 0 : 2] = c;
        tail[f64 ? 1 : 3] = mu;
    }
    __syncthreads();
    for (int i = conv64 + 1 + threadIdx.x; i < m; i += blockDim.x) {
        cp64[i] = tail[0];
        mult64[i] = tail[1];
    }
    for (int i = conv32 + 1 + threadIdx.x; i < m; i += blockDim.x) {
        cp32[i] = split_rn(tail[2]);
        mult32[i] = split_rn(tail[3]);
    }
}

}  // namespace

extern "C" int gp_sweep_noalloc(void *psi_device, const gp_grid *grid, int axis, double h,
                                double dt, int mode, int precision, void *cuda_stream)
{
    if (!psi_device || !grid) return reject(GP_EINVAL, "gp_sweep_noalloc: null argument");
    const bool shape_ok = grid->nx >= 3 && grid->ny >= 3 && (grid->nz == 1 || grid->nz >= 3) &&
                          grid->nx <= GP_MAX_EDGE && grid->ny <= GP_MAX_EDGE &&
                          grid->nz <= GP_MAX_EDGE;
    if (!shape_ok) return reject(GP_EINVAL, "gp_sweep_noalloc: invalid grid");
    if (axis < 0 || axis > 2 || (axis == 2 && grid->nz == 1))
        return reject(GP_EINVAL, "gp_sweep_noalloc: axis must be 0, 1 or (3D only) 2");
    if (!(h > 0) || !(dt > 0) || !std::isfinite(h) || !std::isfinite(dt))
        return reject(GP_EINVAL, "gp_sweep_noalloc: h and dt must be > 0");
    if ((mode != GP_IMAG && mode != GP_REAL) || (precision != GP_C128 && precision != GP_C64))
        return reject(GP_EINVAL, "gp_sweep_noalloc: bad mode or precision");
    const long long points = (long long)grid->nx * grid->ny * grid->nz;
    const size_t elem = precision == GP_C128 ? 16 : 8;
    if ((size_t)points * elem > kScratchBytes)
        return reject(GP_EINVAL, "gp_sweep_noalloc: grid exceeds the static scratch "
                                 "(at most 1048576 complex128 or 2097152 complex64 points)");

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(GP_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(GP_EINTERNAL, "gp_sweep_noalloc: device ordinal out of range");
    if (!g_scratch_addr[dev]) {
        // once per device, with that device current: the device address of
        // the static array (host code cannot use the symbol itself)
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) return reject(GP_ECUDA, "gp_sweep_noalloc: cudaGetSymbolAddress failed");
        g_scratch_addr[dev] = addr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // Forward-elimination tables of (I - kappa L), FP64 with FP32 roundings.
    const int n = axis == 0 ? grid->nx : (axis == 1 ? grid->ny : grid->nz);
    const int m = n - 1;
    const double kap = dt / (4.0 * h * h);
    gp::AxisTables ax;
    ax.n = n;
    ax.h = h;
    gp::fill_tables(ax, m, mode == GP_IMAG ? kap : 0.0, mode == GP_IMAG ? 0.0 : kap, g_cp64, g_mult64,
                    g_cp32, g_mult32);
    unsigned char *tab = base + kScratchBytes;
    ax.cp64 = reinterpret_cast<double2 *>(tab);
    ax.mult64 = ax.cp64 + kTableEntries;
    ax.cp32 = reinterpret_cast<float4 *>(ax.mult64 + kTableEntries);
    ax.mult32 = ax.cp32 + kTableEntries;
    // the host ran the recurrence for the by-value fields (conv, the constant
    // tails, the middle-row multipliers, the window); the device writes the
    // same tables into the static array
    const double kre = ax.kre, kim = ax.kim;
    k_noalloc_tables<<<1, 256, 0, st>>>(m, ax.conv64, ax.conv32, kre, kim, (double)(float)kre,
                                        (double)(float)kim, ax.cp64, ax.mult64, ax.cp32, ax.mult32);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reject(GP_ECUDA, cudaGetErrorString(e));

    gp::SweepGeom g{};
    const long long nx = grid->nx, ny = grid->ny;
    if (axis == 0) { g.n = grid->nx; g.lines_a = grid->ny; g.lines_b = grid->nz; g.stride_a = nx; g.stride_b = nx * ny; g.pstride = 1; }
    else if (axis == 1) { g.n = grid->ny; g.lines_a = grid->nx; g.lines_b = grid->nz; g.stride_a = 1; g.stride_b = nx * ny; g.pstride = nx; }
    else { g.n = grid->nz; g.lines_a = grid->nx; g.lines_b = grid->ny; g.stride_a = 1; g.stride_b = nx; g.pstride = nx * ny; }
    // d' is fully written by the forward pass before the back pass reads it,
    // so the scratch needs no clearing between calls
    e = gp::launch_sweep_yz(precision, mode, psi_device, base, ax, g, nullptr, st);
    if (e != cudaSuccess) return reject(GP_ECUDA, cudaGetErrorString(e));
    return GP_OK;
}
