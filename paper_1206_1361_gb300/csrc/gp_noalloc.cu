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
double2 g_cp64[kTableEntries], g_mult64[kTableEntries];
float4 g_cp32[kTableEntries], g_mult32[kTableEntries];

int reject(int code, const char *msg)
{
    gp::set_thread_error(msg);
    return code;
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
    // pageable sources: each copy returns once its bytes are staged
    const struct { void *dst; const void *src; size_t bytes; } copies[4] = {
        {ax.cp64, g_cp64, m * sizeof(double2)}, {ax.mult64, g_mult64, m * sizeof(double2)},
        {ax.cp32, g_cp32, m * sizeof(float4)}, {ax.mult32, g_mult32, m * sizeof(float4)}};
    for (const auto &cp : copies) {
        e = cudaMemcpyAsync(cp.dst, cp.src, cp.bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return reject(GP_ECUDA, cudaGetErrorString(e));
    }

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
