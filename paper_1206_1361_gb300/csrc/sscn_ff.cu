// sscn_ff.cu -- the FP64-class form of the Crank-Nicolson sweeps (calclux,
// calcluy, calcluz, with calcnu fused into the x sweep) in float-float
// arithmetic on the FP32 pipe, sm_103a.
//
// GB300 executes FP64 at 2 multiply-adds per clock per SM against 128 for
// FP32, so FP64 sweeps are bound by the FP64 pipe at a small fraction of the
// HBM bandwidth.  This form carries psi and every recurrence as float-float
// values (hi + lo, ~48 significant bits; sscn_ff.cuh), which keeps the
// result within the FP64 tolerances while the sweeps run on the FP32 pipe.
//
// The pipeline is the TMA-staged one of the complex64 sweeps: one CTA owns a
// tile of L = 32 K lines (one consumer thread per line), a producer warp
// streams chunks of C = 8 points of all L lines through an S-stage
// shared-memory ring (cp.async.bulk.tensor, one mbarrier per stage) and
// stores finished chunks back with TMA stores.  Each consumer runs the
// forward elimination of its line, (I - kappa L) v = psi,
//     d'_i = (psi_i + kappa d'_{i-1}) mult_i,
// keeps d' for the last two chunks in shared memory, and back-substitutes
// over a window: the values of chunk q-1 are produced after the forward pass
// of chunk q, from v ~ d' at W points into chunk q,
//     v_i = d'_i - c'_i v_{i+1},   u_i = 2 v_i - psi_i,
// which is the Crank-Nicolson update (I + kappa L) = 2 I - (I - kappa L).
// The dropped term decays as |c'|^(W+1); the host picks W <= C with
// max|c'|^(W+1) < 2^-50, below the float-float rounding.  The last chunks
// are back-substituted exactly from v_m = d'_m.
//
// calcnu (real time): psi <- P_x[i] P_y[j] P_z[k] (1 + delta) psi with the
// unit-modulus factor tables P_k = exp(-i dt omega_k^2 x^2 / 2) and
// delta = exp(-i a) - 1, a = G |psi|^2 (G the integral of g over the step),
// from its Taylor series for |a| < 2^-8 (first dropped terms below 2^-57)
// and through FP64 sincos beyond.  Imaginary time: the real factor
// s P_x P_y P_z (1 + eps), eps = exp(-a) - 1, a = G s^2 |psi|^2, s the
// pending renormalisation scale.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "sscn_ff.cuh"
#include "sscn_internal.h"
#include "sscn_tma.cuh"

namespace gp {
namespace {

using namespace gp::tma;
using namespace gp::ff;

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per chunk wait
constexpr int kErrTimeout = 2;
constexpr int kC = 8;                              // points per chunk (128-byte x rows)

struct FfArgs {
    int n;                  // stored points per line (m = n - 1 unknowns)
    int lines_a;            // extent of the in-tile line index
    int win, conv;          // window W (1 .. C), first constant table index
    int win32;              // the window's first steps that run in FP32 (0 .. W - 1)
    FfCoef cinf, minf;      // the constants past conv
    const FfCoef *cp, *mult;
    float2 kk_hi, kk_lo;    // kappa per lane: (k, k) imaginary, (-k, k) real time
    const FfCoef *px;       // calcnu (x sweep)
    const double2 *py, *pz;
    StepG g;
    const double *scale;
    double *partials;       // norm partials (NORM)
    int *err;
};

__device__ __forceinline__ C ld(const unsigned char *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return C{f2(v.x, v.y), f2(v.z, v.w)};
}
// point c of a chunk loaded whole from tensor memory (tmem_ld32)
#define GP_FF_FROM(w, c) C{f2((w)[4 * (c)], (w)[4 * (c) + 1]), f2((w)[4 * (c) + 2], (w)[4 * (c) + 3])}

__device__ __forceinline__ void st(unsigned char *p, C z)
{
    *reinterpret_cast<float4 *>(p) = make_float4(z.hi.x, z.hi.y, z.lo.x, z.lo.y);
}

// Crank-Nicolson line steps.  MODE 0: kappa = k, real tables.  MODE 1:
// kappa = i k, complex tables.
template <int MODE> struct FfLine {
    float2 kh, kl;
    // (p + kappa d) mult
    __device__ __forceinline__ C fwd(C p, C d, const FfCoef &f) const
    {
        if (MODE == 0) return rmul(add(p, lmul(d, kh, kl)), f);
        return cmul(add(p, imul(d, kh, kl)), f);
    }
    // d - c' v
    __device__ __forceinline__ C back(C d, const FfCoef &c, C v) const
    {
        if (MODE == 0) return sub(d, rmul(v, c));
        return sub(d, cmul(v, c));
    }
    // d - c' v on the hi parts alone (FP32): the first steps of a window,
    // whose rounding the remaining steps damp below the float-float
    // rounding before any result is kept
    __device__ __forceinline__ C back32(C d, const FfCoef &c, C v) const
    {
        float2 r = fma2(neg(c.rh), v.hi, d.hi);
        if (MODE != 0) r = fma2(neg(c.ih), swap(v.hi), r);
        return C{r, f2(0.f, 0.f)};
    }
};

// calcnu at one point of an x line (see the file comment).
template <int MODE> struct FfCalcnu {
    const FfCoef *px;
    FfCoef pyz;          // P_y[j] P_z[k] (times s in imaginary time), expanded
    float2 acoef;        // G (times s^2 in imaginary time)
    float2 fyz;          // imaginary time: s P_y[j] P_z[k] as a scalar pair

    __device__ __forceinline__ void setup(const FfArgs &a, int j, int k)
    {
        px = a.px;
        const double2 y = a.py[j], z = a.pz[k];
        const double G = a.g.value();
        if (MODE == 0) {
            const double s = a.scale ? *a.scale : 1.0;
            const double f = s * y.x * z.x;
            fyz = split(f);
            acoef = split(G * s * s);
            pyz = expand(f, 0.0);
        } else {
            pyz = expand(y.x * z.x - y.y * z.y, y.x * z.y + y.y * z.x);
            acoef = split(G);
            fyz = f2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ C apply(C p, int i) const
    {
        const float2 a = s_mul(acoef, abs2(p));
        if (MODE == 0) {
            // eps = exp(-a) - 1 = -a + a^2/2 - a^3/6 + a^4/24 - a^5/120 + ...
            float2 eps;
            if (fabsf(a.x) < 0x1p-8f) {
                const float q = __fmul_rn(a.x, a.x);
                float qe = fmaf(a.x, a.x, -q);
                qe = fmaf(2.f * a.x, a.y, qe);
                eps = s_two_sum(-a.x, 0.5f * q);
                const float tail = fmaf(q, fmaf(a.x, -1.f / 120, 1.f / 24) * q, -a.x * q * (1.f / 6));
                eps = s_norm(f2(eps.x, eps.y + ((0.5f * qe - a.y) + tail)));
            } else {
                eps = split(expm1(-join(a)));
            }
            const FfCoef &x = px[i];
            const float2 f = s_mul(fyz, f2(x.rh.x, x.rl.x));
            const float2 F = s_norm(s_add(f, s_mul(f, eps)));
            return norm(lmul(p, f2(F.x, F.x), f2(F.y, F.y)));
        }
        // delta = exp(-i a) - 1 = (cos a - 1) - i sin a
        float2 dr, di;
        if (fabsf(a.x) < 0x1p-8f) {
            const float q = __fmul_rn(a.x, a.x);
            float qe = fmaf(a.x, a.x, -q);
            qe = fmaf(2.f * a.x, a.y, qe);
            // cos a - 1 = -a^2/2 + a^4/24 - ...   (a^6/720 < 2^-57)
            dr = f2(-0.5f * q, fmaf(q * q, 1.f / 24, -0.5f * qe));
            // -sin a = -a + a^3/6 - a^5/120 + ...  (a^7/5040 < 2^-68)
            di = f2(-a.x, fmaf(a.x * q, fmaf(q, -1.f / 120, 1.f / 6), -a.y));
        } else {
            double sh, ch;
            sincos(0.5 * join(a), &sh, &ch);
            dr = split(-2.0 * sh * sh);
            di = split(-2.0 * sh * ch);
        }
        const FfCoef D{f2(dr.x, dr.x), f2(dr.y, dr.y), f2(-di.x, di.x), f2(-di.y, di.y)};
        const C q2 = cmul(cmul(p, px[i]), pyz);
        return norm(add(q2, cmul(q2, D)));
    }
};

template <int L, int AXIS> struct FfTile {
    static constexpr int E = 16;
    static constexpr int kStageBytes = L * kC * E;
    static __device__ __forceinline__ int off(int l, int c)
    {
        if (AXIS == 0) return l * (kC * E) + ((c ^ (l & 7)) << 4);   // 128-byte swizzle
        return (c * L + l) * E;
    }
};

// Columns of tensor memory a CTA of the TMEM-ring shapes allocates: d' of
// two chunks of C points, 4 FP32 words (re hi, im hi, re lo, im lo) each.
constexpr int kTmemCols = 2 * kC * 4;

template <int K, int S, bool TM>
constexpr size_t ff_smem_bytes()
{
    constexpr size_t L = 32 * K;
    return 1024 + (size_t)S * L * kC * 16 + (TM ? 0 : 2 * (size_t)kC * L * 16) +
           2 * S * sizeof(uint64_t) + 32 * sizeof(double) + 16;
}

// Resident CTAs per SM the TMEM shapes are built for: as many as shared
// memory admits, at most 512 / kTmemCols (the columns of one SM).
template <int K, int S, bool TM>
constexpr int ff_min_blocks()
{
    if (!TM) return 1;
    constexpr int by_smem = (int)((227 * 1024) / ff_smem_bytes<K, S, TM>());
    constexpr int by_tmem = 512 / kTmemCols;
    return by_smem < by_tmem ? by_smem : by_tmem;
}

// Warp-specialised CTA: K consumer warps own L = 32 K lines; warp K is the
// producer, whose lane 0 issues every TMA load and store.  full[s] completes
// when a chunk has landed, ready[s] when all K consumer warps have written
// the chunk's final values; the producer stores a ready chunk and reuses its
// stage once the store has read shared memory.
// TM: the d' ring lives in tensor memory (each consumer thread's line in
// its TMEM lane), which leaves shared memory to the stages and so admits
// more resident CTAs; every lane of a consumer warp then runs the same
// instruction stream (the tcgen05 accesses are warp-wide), lanes past the
// end of a ragged tile computing on the zeros TMA filled in, whose rows the
// TMA store clips.
template <int MODE, int AXIS, bool NL, bool NORM, int K, int S, bool TM>
__global__ void __launch_bounds__(32 * (K + 1), ff_min_blocks<K, S, TM>())
k_sweep_ff(const __grid_constant__ CUtensorMap map, const FfArgs args)
{
    constexpr int L = 32 * K;
    constexpr int Cc = kC;
    using G = FfTile<L, AXIS>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *stages = smem;
    float4 *ring = reinterpret_cast<float4 *>(stages + S * G::kStageBytes);   // [2][C][L]
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (TM ? 0 : 2 * Cc * L));
    uint64_t *ready = full + S;
    double *red = reinterpret_cast<double *>(ready + S);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(red + 32);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == K;
    const int l = producer ? 0 : threadIdx.x;
    const int tile0 = blockIdx.x * L;
    const int a = tile0 + l;
    const bool active = !producer && a < args.lines_a;
    const bool run = TM ? !producer : active;       // computes (see TM above)
    const int m = args.n - 1;
    const int Q = (args.n + Cc - 1) / Cc;
    const int conv = args.conv, win = args.win;

    auto coords = [&](int q, int &c0, int &c1, int &c2) {
        if (AXIS == 0) { c0 = q * Cc * 2; c1 = tile0; c2 = blockIdx.y; }
        else if (AXIS == 1) { c0 = tile0 * 2; c1 = q * Cc; c2 = blockIdx.y; }
        else { c0 = tile0 * 2; c1 = blockIdx.y; c2 = q * Cc; }
    };
    auto stage_ptr = [&](int q) { return stages + (q % S) * G::kStageBytes; };
    auto at = [&](int q, int c) { return stage_ptr(q) + G::off(l, c); };

    if (TM && warp == 0) {
        tmem_alloc(tslot, kTmemCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], K);
        }
        fence_mbar_init();
    }
    if (TM) tmem_fence_before();
    __syncthreads();
    if (TM) tmem_fence_after();
    // this warp's TMEM lanes (consumer warps 0 .. K-1 reach lanes 32 (w % 4) ..)
    const uint32_t tbase = TM ? *tslot + ((uint32_t)(32 * (warp & 3)) << 16) : 0u;

    bool failed = false;
    float2 nacc = f2(0.f, 0.f);        // float-float sum of |u|^2 (NORM)
    if (producer) {
        if (lane == 0) {
            auto store = [&](int q) {
                int c0, c1, c2;
                coords(q, c0, c1, c2);
                tma_store_3d(&map, stage_ptr(q), c0, c1, c2);
                bulk_commit();
            };
            for (int q = 0; q < Q && !failed; ++q) {
                if (q >= S) {
                    const int o = q - S;
                    if (!mbar_wait_bounded(&ready[o % S], (uint32_t)((o / S) & 1), kWaitLimitNs)) {
                        failed = true;
                        break;
                    }
                    store(o);
                    bulk_wait_read<0>();
                }
                int c0, c1, c2;
                coords(q, c0, c1, c2);
                mbar_arrive_expect_tx(&full[q % S], G::kStageBytes);
                tma_load_3d(stage_ptr(q), &map, &full[q % S], c0, c1, c2);
            }
            for (int o = Q > S ? Q - S : 0; o < Q && !failed; ++o) {
                if (!mbar_wait_bounded(&ready[o % S], (uint32_t)((o / S) & 1), kWaitLimitNs)) {
                    failed = true;
                    break;
                }
                store(o);
            }
            bulk_wait_all();
        }
    } else {
        const FfLine<MODE> cn{args.kk_hi, args.kk_lo};
        const int win32 = args.win32;
        FfCalcnu<MODE> nl;
        // lanes past a ragged tile's end take the last line's factors
        if (NL && run) nl.setup(args, active ? a : args.lines_a - 1, blockIdx.y);
        auto cp = [&](int t) -> FfCoef { return t < conv ? args.cp[t] : args.cinf; };
        auto mult = [&](int t) -> FfCoef { return t < conv ? args.mult[t] : args.minf; };
        auto slot = [&](int i) -> float4 * {
            return ring + ((i / Cc) & 1) * Cc * L + (i % Cc) * L + l;
        };
        // TMEM column of point i: chunk parity, then 4 words per point
        auto tcol = [&](int i) -> uint32_t { return (uint32_t)((((i / Cc) & 1) * Cc + i % Cc) * 4); };
        auto put = [&](int i, C d) {
            if (TM) tmem_st4(tbase + tcol(i), d.hi.x, d.hi.y, d.lo.x, d.lo.y);
            else *slot(i) = make_float4(d.hi.x, d.hi.y, d.lo.x, d.lo.y);
        };
        auto get = [&](int i) -> C {
            const float4 v = TM ? tmem_ld4(tbase + tcol(i)) : *slot(i);
            return C{f2(v.x, v.y), f2(v.z, v.w)};
        };
        auto acc_norm = [&](C u) {
            if (NORM && active) nacc = s_norm(s_add(nacc, abs2(u)));
        };
        auto output = [&](C v, unsigned char *tile_slot) {
            const C u = twice_minus(v, ld(tile_slot));
            st(tile_slot, u);
            acc_norm(u);
        };
        C d = cz();
        for (int q = 0; q < Q; ++q) {
            bool ok = mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kWaitLimitNs);
            if (TM) ok = __all_sync(0xffffffffu, ok);    // the warp leaves together
            if (!ok) {
                failed = true;
                break;
            }
            const bool last = q == Q - 1;
            const bool fast = run && q >= 2 && !last && (q - 1) * Cc - 1 >= conv &&
                              (q + 1) * Cc - 1 <= m;
            if (fast) {
                // interior chunk: every point an unknown, constant tables
                const FfCoef minf = args.minf, cinf = args.cinf;
                auto fwd_at = [&](int c) {
                    unsigned char *tc = at(q, c);
                    C p = ld(tc);
                    if (NL) {
                        p = nl.apply(p, q * Cc + c);
                        st(tc, p);
                    }
                    d = cn.fwd(p, d, minf);
                    put(q * Cc + c, d);
                };
                if constexpr (NL) {
                    // with calcnu, unrolled by 4 (1.7 % faster than by 8)
#pragma unroll 4
                    for (int c = 0; c < Cc; ++c) fwd_at(c);
                } else {
#pragma unroll
                    for (int c = 0; c < Cc; ++c) fwd_at(c);
                }
                if constexpr (TM) {
                    // window: the seed d'_{W-1} by its own load (a runtime
                    // column), then back through the chunk's points W-2 .. 0
                    C v = get(q * Cc + win - 1);
                    {
                        float w[32];
                        tmem_ld32(tbase + tcol(q * Cc), w);
#pragma unroll
                        for (int c = Cc - 2; c >= 0; --c) {
                            if (c > win - 2) continue;
                            if (c >= win - 1 - win32) v = cn.back32(GP_FF_FROM(w, c), cinf, v);
                            else v = cn.back(GP_FF_FROM(w, c), cinf, v);
                        }
                    }
                    float w[32];
                    tmem_ld32(tbase + tcol((q - 1) * Cc), w);
#pragma unroll
                    for (int c = Cc - 1; c >= 0; --c) {
                        v = cn.back(GP_FF_FROM(w, c), cinf, v);
                        output(v, at(q - 1, c));
                    }
                } else {
                    C v = get(q * Cc + win - 1);
                    for (int c = win - 2; c >= 0; --c)
                        v = c >= win - 1 - win32 ? cn.back32(get(q * Cc + c), cinf, v)
                                                 : cn.back(get(q * Cc + c), cinf, v);
#pragma unroll
                    for (int c = Cc - 1; c >= 0; --c) {
                        v = cn.back(get((q - 1) * Cc + c), cinf, v);
                        output(v, at(q - 1, c));
                    }
                }
            } else {
                if (run) {
#pragma unroll 2
                    for (int c = 0; c < Cc; ++c) {
                        const int j = q * Cc + c;
                        if (j >= 1 && j <= m) {
                            C p = ld(at(q, c));
                            if (NL) {
                                p = nl.apply(p, j);
                                st(at(q, c), p);
                            }
                            d = cn.fwd(p, d, mult(j - 1));
                            put(j, d);
                        }
                    }
                }
                if (run) {
                    if (!last && q >= 1) {
                        C v = get(q * Cc + win - 1);
                        for (int c = win - 2; c >= 0; --c) v = cn.back(get(q * Cc + c), cp(q * Cc + c - 1), v);
                        for (int c = Cc - 1; c >= 0; --c) {
                            const int i = (q - 1) * Cc + c;
                            if (i < 1) break;
                            v = cn.back(get(i), cp(i - 1), v);
                            output(v, at(q - 1, c));
                        }
                    } else if (last) {
                        C v = d;
                        const int lo = q >= 1 ? (q - 1) * Cc : 0;
                        for (int i = m; i >= lo && i >= 1; --i) {
                            if (i < m) v = cn.back(get(i), cp(i - 1), v);
                            output(v, at(i / Cc, i % Cc));
                        }
                    }
                }
            }
            if (q >= 1 || last) {
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    if (q >= 1) mbar_arrive(&ready[(q - 1) % S]);
                    if (last) mbar_arrive(&ready[q % S]);
                }
            }
        }
    }
    if (failed) atomicOr(args.err, kErrTimeout);
    if (TM) {
        // every warp is done with tensor memory before it is released
        if (!producer) tmem_wait_st();
        tmem_fence_before();
        __syncthreads();
        if (warp == 0) {
            tmem_fence_after();
            tmem_dealloc(*tslot, kTmemCols);
        }
    }
    if (NORM) {
        double v = join(nacc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            double r = lane < K ? red[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
            if (lane == 0) args.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = r;
        }
    }
}

template <int MODE, int AXIS, bool NL, bool NORM, int K, int S, bool TM>
cudaError_t launch_inst(const CUtensorMap &map, const FfArgs &args, int tiles, int lines_b,
                        cudaStream_t st)
{
    auto kern = k_sweep_ff<MODE, AXIS, NL, NORM, K, S, TM>;
    static size_t smem_of[64] = {};           // per device ordinal, 0: not configured
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!smem_of[dev]) {
        size_t smem = ff_smem_bytes<K, S, TM>();
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // TM: no more resident CTAs than one SM's tensor memory holds (an
        // allocation beyond it would wait for another CTA to finish), so
        // pad the shared memory until the occupancy says so
        for (;;) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            if (!TM) break;
            int blocks = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * (K + 1), smem);
            if (e != cudaSuccess) return e;
            if (blocks * kTmemCols <= 512) break;
            smem += 1024;
            if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        }
        smem_of[dev] = smem;
    }
    kern<<<dim3(tiles, lines_b), 32 * (K + 1), smem_of[dev], st>>>(map, args);
    return cudaGetLastError();
}

template <int AXIS, int K, int S, bool TM>
cudaError_t launch_axis(int mode, bool nl, bool norm, const CUtensorMap &map, const FfArgs &args,
                        int tiles, int lines_b, cudaStream_t st)
{
    // calcnu rides on the x sweep only
    if (nl && AXIS != 0) return cudaErrorInvalidValue;
#define GP_FF(MODE, NLV, NORMV) \
    return launch_inst<MODE, AXIS, (NLV && AXIS == 0), NORMV, K, S, TM>(map, args, tiles, lines_b, st)
    if (mode == 0) {
        if (nl) { if (norm) GP_FF(0, true, true); GP_FF(0, true, false); }
        if (norm) GP_FF(0, false, true);
        GP_FF(0, false, false);
    }
    if (nl) { if (norm) GP_FF(1, true, true); GP_FF(1, true, false); }
    if (norm) GP_FF(1, false, true);
    GP_FF(1, false, false);
#undef GP_FF
}

// Tile shapes (consumer warps K, stages S, d' ring in tensor memory); a CTA
// owns 32 K lines.  Index 0 is the default: the fastest measured at 256^3
// (4 consumer warps, 3 stages, TMEM ring: 4 CTAs and 16 consumer warps per
// SM, against 5 CTAs and 10 consumer warps with the ring in shared memory).
struct Shape { int K, S; bool TM; };
constexpr Shape kShapes[] = {{4, 3, true},  {2, 3, true},  {2, 4, true}, {2, 3, false},
                             {1, 4, false}, {2, 4, false}, {4, 3, false}};
constexpr int kNumShapes = 7;

template <int K, int S, bool TM>
cudaError_t launch_shape(int mode, int axis, bool nl, bool norm, const CUtensorMap &map,
                         const FfArgs &args, int tiles, int lines_b, cudaStream_t st)
{
    if (axis == 0) return launch_axis<0, K, S, TM>(mode, nl, norm, map, args, tiles, lines_b, st);
    if (axis == 1) return launch_axis<1, K, S, TM>(mode, nl, norm, map, args, tiles, lines_b, st);
    return launch_axis<2, K, S, TM>(mode, nl, norm, map, args, tiles, lines_b, st);
}

Shape shape_of(int s) { return kShapes[s < 0 || s >= kNumShapes ? 0 : s]; }

// --------------------------------------------------------------- conversions

__global__ void k_ff_from_c128(float4 *__restrict__ dst, const double2 *__restrict__ src,
                               long long count, const double *scale)
{
    const double s = scale ? *scale : 1.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        const float2 r = split(s * v.x), im = split(s * v.y);
        dst[i] = make_float4(r.x, im.x, r.y, im.y);
    }
}

__global__ void k_ff_set_one(double *x) { *x = 1.0; }

// split(v) -- hi = v rounded to FP32, lo = v - hi (exact in FP64) rounded to
// FP32 -- from the bits of v with integer and FP32 operations only: the grid
// conversion streams whole grids, and GB300 runs FP64 arithmetic and FP64
// conversions on its narrow FP64 pipe.  With v = s m 2^(e-52) (m the 53-bit
// significand) and -97 <= e <= 126, hi = s r 2^(e-23) for r = m / 2^29
// rounded to nearest, ties to even, and v - hi = s d 2^(e-52) with the
// integer d = m - r 2^29, |d| <= 2^28: lo = RN(s d) 2^-52 2^e, whose two
// power-of-two scalings are exact (a subnormal lo is a multiple of 2^-149,
// and then |d| < 2^24): bit-identical to split.
__device__ __forceinline__ float2 split_bits_normal(unsigned long long b, int e)
{
    const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
    unsigned long long r = m >> 29;
    const unsigned long long rem = m & 0x1fffffffull;
    if (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1ull))) ++r;
    const int d = (int)((long long)m - (long long)(r << 29));
    int eh = e;
    if (r == 0x1000000ull) {        // rounded up to the next power of two
        r >>= 1;
        ++eh;
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const float hi = __uint_as_float(sign | ((unsigned)(eh + 127) << 23) | ((unsigned)r & 0x7fffffu));
    // (the sign on d: an exact remainder of zero gives lo = +0, as v - hi does)
    const float lo = __int2float_rn(sign ? -d : d) * 0x1p-52f * __uint_as_float((unsigned)(e + 127) << 23);
    return f2(hi, lo);
}

// split(v) for every v: bit-identical for 2^-97 <= |v| < 2^127 (above, where
// hi may overflow, it calls split).  Below 2^-97 -- far under anything the
// float-float sweeps resolve next to an O(1) state -- it splits 2^100 v and
// scales both halves back in FP32, each rounded once more into FP32's
// subnormal range (within 2^-147 of v), and below 2^-180 it returns zeros
// carrying the sign of v, as split does.
__device__ __forceinline__ float2 split_bits(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e > 126) return split(v);
    if (e >= -97) return split_bits_normal(b, e);
    if (e < -180) {
        const float z = (b >> 63) ? -0.f : 0.f;
        return f2(z, z);
    }
    const float2 t = split_bits_normal(b + (100ull << 52), e + 100);
    return f2(t.x * 0x1p-100f, t.y * 0x1p-100f);
}

// complex128 psi of an nx * ny * nz grid into pairs, the Dirichlet nodes
// (index 0 of each bounded axis) set to zero: blocks walk groups of kFromLines
// x-lines, threads the points of a line, each thread's loads of the group's
// lines issued together.  A line's (j, k) is found once per group (a 64-bit
// division per point, with one load in flight per thread, held this pass to
// 2 TB/s).
constexpr int kFromLines = 4;
__global__ void k_ff_from_c128_grid(float4 *__restrict__ dst, const double2 *__restrict__ src, int nx,
                                    int ny, int nz)
{
    const int lines = ny * nz;             // <= 8192^2
    for (int l0 = blockIdx.x * kFromLines; l0 < lines; l0 += gridDim.x * kFromLines) {
        bool keep[kFromLines];             // line inside the grid and off the Dirichlet planes
        int j = l0 % ny, k = l0 / ny;
#pragma unroll
        for (int u = 0; u < kFromLines; ++u) {
            keep[u] = l0 + u < lines && j > 0 && (nz == 1 || k > 0);
            if (++j == ny) {
                j = 0;
                ++k;
            }
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double2 v[kFromLines];
#pragma unroll
            for (int u = 0; u < kFromLines; ++u)
                v[u] = l0 + u < lines ? src[(long long)(l0 + u) * nx + i] : make_double2(0.0, 0.0);
#pragma unroll
            for (int u = 0; u < kFromLines; ++u) {
                if (l0 + u >= lines) break;
                float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i > 0 && keep[u]) {
                    const float2 r = split_bits(v[u].x), im = split_bits(v[u].y);
                    o = make_float4(r.x, im.x, r.y, im.y);
                }
                dst[(long long)(l0 + u) * nx + i] = o;
            }
        }
    }
}

__global__ void k_ff_to_c128(double2 *__restrict__ dst, const float4 *__restrict__ src,
                             long long count, const double *scale)
{
    const double s = scale ? *scale : 1.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        dst[i] = make_double2(s * ((double)v.x + (double)v.z), s * ((double)v.y + (double)v.w));
    }
}

// --------------------------------------------------------------- observables
//
// A thread owns one x and walks a chunk of kObsLines consecutive y-lines of
// one plane (blocks over x segments, line chunks and planes; coalesced
// 16-byte loads of the pairs): each point is loaded once as the thread's own
// value and carried to the next line as that line's y-neighbour; the
// x-neighbour comes from the next lane (lane 31 loads it), the z-neighbour
// from the next plane, which that plane's blocks, resident at the same time,
// find in L2.  Per point: a = |psi|^2, a^2, y_j^2 a, V_y(j) a and the
// neighbour terms R = Re(psi_next conj(psi)) along x, y, z (zero beyond the
// last stored point), each a float-float product summed per thread in
// float-float (TwoSum + Fast2Sum after every addition); the factors constant
// for the thread (x^2, V_x) or the block (z^2, V_z) multiply its sum of a
// once.  Warp sums combine the same way, the block's in FP64, and each
// block writes one 9-wide FP64 row of the FP64 observables (the finish forms
// K = 2 S0 - 2 R), so the rows and the fixed-order finish are shared with
// the other forms.
__device__ __forceinline__ float2 lane_sum(C z)
{
    const float2 s = s_two_sum(z.hi.x, z.hi.y);
    return f2(s.x, s.y + (z.lo.x + z.lo.y));
}

__global__ void __launch_bounds__(256)
k_observables_ff(const float4 *__restrict__ psi, ObsArgs a, const float2 *__restrict__ x2ff,
                 const float2 *__restrict__ vxff, double *__restrict__ rows)
{
    __shared__ float2 yt[2][kObsLines];
    __shared__ double red[8][8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = blockIdx.y * kObsLines, j1 = min(j0 + kObsLines, ny);
    const int k = blockIdx.z;
    for (int t = threadIdx.x; t < kObsLines && j0 + t < ny; t += blockDim.x) {
        yt[0][t] = split(a.y2[j0 + t]);
        yt[1][t] = split(a.vy[j0 + t]);
    }
    __syncthreads();
    const bool in = i < nx, has_z = nz > 1 && k + 1 < nz;
    const long long plane = (long long)nx * ny;
    const float4 *pk = psi + k * plane;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    auto cv = [](float4 v) { return C{f2(v.x, v.y), f2(v.z, v.w)}; };
    float2 acc[7];                          // S0, Sy, SVy, S4, Rx, Ry, Rz
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] = f2(0.f, 0.f);
    auto put = [&](int q, float2 t) { acc[q] = s_norm(s_add(acc[q], t)); };
    float4 v4 = in ? pk[(long long)j0 * nx + i] : zero;
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        const long long at = (long long)j * nx + i;
        const float4 vn4 = (in && j + 1 < ny) ? pk[at + nx] : zero;      // y-neighbour
        const float4 vz4 = (in && has_z) ? pk[at + plane] : zero;        // z-neighbour
        float4 nb4;                                                      // x-neighbour
        nb4.x = __shfl_down_sync(0xffffffffu, v4.x, 1);
        nb4.y = __shfl_down_sync(0xffffffffu, v4.y, 1);
        nb4.z = __shfl_down_sync(0xffffffffu, v4.z, 1);
        nb4.w = __shfl_down_sync(0xffffffffu, v4.w, 1);
        if (lane == 31) nb4 = (i + 1 < nx) ? pk[at + 1] : zero;
        const C v = cv(v4);
        const float2 am = abs2(v);
        put(0, am);
        put(1, s_mul(yt[0][j - j0], am));
        put(2, s_mul(yt[1][j - j0], am));
        put(3, s_mul(am, am));
        put(4, lane_sum(lmul(cv(nb4), v.hi, v.lo)));
        put(5, lane_sum(lmul(cv(vn4), v.hi, v.lo)));
        if (nz > 1) put(6, lane_sum(lmul(cv(vz4), v.hi, v.lo)));
        v4 = vn4;
    }
    // S0, Sx, Sy, SVx + SVy, S4, Rx, Ry, Rz
    const float2 x2 = in ? x2ff[i] : f2(0.f, 0.f), vx = in ? vxff[i] : f2(0.f, 0.f);
    float2 t8[8] = {acc[0], s_mul(x2, acc[0]), acc[1], s_norm(s_add(s_mul(vx, acc[0]), acc[2])),
                    acc[3], acc[4], acc[5], acc[6]};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float2 t = f2(__shfl_down_sync(0xffffffffu, t8[q].x, o),
                                __shfl_down_sync(0xffffffffu, t8[q].y, o));
            t8[q] = s_norm(s_add(t8[q], t));
        }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[wib][q] = join(t8[q]);
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][threadIdx.x];
        red[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sc = *a.scale, s2 = sc * sc;
        const double *t = red[0];
        double *out = rows + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x * kObsWidth +
                      (long long)blockIdx.x * kObsWidth;
        out[0] = s2 * t[0];
        out[1] = s2 * t[1];
        out[2] = s2 * t[2];
        out[3] = s2 * a.z2[k] * t[0];
        out[4] = s2 * (t[3] + a.vz[k] * t[0]);
        out[5] = s2 * s2 * t[4];
        out[6] = s2 * t[5];
        out[7] = s2 * t[6];
        out[8] = s2 * t[7];
    }
}

int point_blocks(long long count)
{
    const long long b = (count + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

FfCoef ff_expand(double2 v)
{
    const float rh = (float)v.x, ih = (float)v.y;
    const float rl = (float)(v.x - (double)rh), il = (float)(v.y - (double)ih);
    return FfCoef{make_float2(rh, rh), make_float2(rl, rl), make_float2(-ih, ih), make_float2(-il, il)};
}

void ff_tables(int m, const double2 *cp64, const double2 *mult64, int conv64, double cmax,
               double k, int chunk, FfAxis &out, FfCoef *cp, FfCoef *mult)
{
    for (int i = 0; i < m; ++i) {
        cp[i] = ff_expand(cp64[i]);
        mult[i] = ff_expand(mult64[i]);
    }
    out.n = m + 1;
    out.conv = conv64;
    out.cinf = cp[m - 1];
    out.minf = mult[m - 1];
    out.k = k;
    // window: smallest W <= chunk with cmax^(W+1) < 2^-50
    out.win = 0;
    double p = cmax;
    for (int w = 1; w <= chunk; ++w) {
        p *= cmax;
        if (p < 0x1p-50) {
            out.win = w;
            break;
        }
    }
    // FP32 window steps: an error of 2^-24 made at window step s (s = 1 ..
    // W - 1 from the seed, whose lo part those steps drop) passes W - s more
    // steps, each scaling it by at most cmax, before the first result: it
    // stays below 2^-50 when cmax^(W - s) < 2^-26
    int kmin = 1;
    for (double q = cmax; q >= 0x1p-26 && kmin <= 64; q *= cmax) ++kmin;
    out.win32 = out.win > 0 ? std::max(0, std::min(out.win - 1, out.win - kmin)) : 0;
}

int ff_shapes() { return kNumShapes; }
int ff_chunk(int) { return kC; }

int ff_blocks(int shape, const SweepGeom &g)
{
    const int L = 32 * shape_of(shape).K;
    return ((g.lines_a + L - 1) / L) * g.lines_b;
}

cudaError_t make_ff_map(int shape, void *psi, int nx, int ny, int nz, int axis, CUtensorMap *out)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Shape sh = shape_of(shape);
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * nx * 8, (cuuint64_t)2 * nx * ny * 8};
    cuuint32_t box[3];
    CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    const int L = 32 * sh.K;
    if (axis == 0) { box[0] = 2 * kC; box[1] = L; box[2] = 1; sw = CU_TENSOR_MAP_SWIZZLE_128B; }
    else if (axis == 1) { box[0] = 2 * L; box[1] = kC; box[2] = 1; }
    else { box[0] = 2 * L; box[1] = 1; box[2] = kC; }
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, psi, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_sweep_ff(int shape, int mode, int axis, const CUtensorMap &map,
                            const FfAxis &ax, const SweepGeom &g, const FfNonlin *nl,
                            const Partials *norm_out, int *err, cudaStream_t st)
{
    if (ax.win < 1 || ax.win > kC) return cudaErrorInvalidValue;
    FfArgs args{};
    args.n = g.n;
    args.lines_a = g.lines_a;
    args.win = ax.win;
    args.win32 = ax.win32;
    args.conv = ax.conv;
    args.cinf = ax.cinf;
    args.minf = ax.minf;
    args.cp = ax.cp;
    args.mult = ax.mult;
    const float kh = (float)ax.k, kl = (float)(ax.k - (double)kh);
    if (mode == 0) {
        args.kk_hi = make_float2(kh, kh);
        args.kk_lo = make_float2(kl, kl);
    } else {
        args.kk_hi = make_float2(-kh, kh);
        args.kk_lo = make_float2(-kl, kl);
    }
    if (nl) {
        args.px = nl->px;
        args.py = nl->py;
        args.pz = nl->pz;
        args.g = nl->g;
        args.scale = nl->scale;
    }
    args.partials = norm_out ? norm_out->buf : nullptr;
    args.err = err;
    const Shape sh = shape_of(shape);
    const int tiles = (g.lines_a + 32 * sh.K - 1) / (32 * sh.K);
    const bool has_nl = nl != nullptr, norm = norm_out != nullptr;
    const int lb = g.lines_b;
#define GP_FF_SHAPE(I) \
    launch_shape<kShapes[I].K, kShapes[I].S, kShapes[I].TM>(mode, axis, has_nl, norm, map, args, tiles, lb, st)
    switch (shape) {
    case 1: return GP_FF_SHAPE(1);
    case 2: return GP_FF_SHAPE(2);
    case 3: return GP_FF_SHAPE(3);
    case 4: return GP_FF_SHAPE(4);
    case 5: return GP_FF_SHAPE(5);
    case 6: return GP_FF_SHAPE(6);
    default: return GP_FF_SHAPE(0);
    }
#undef GP_FF_SHAPE
}

cudaError_t launch_ff_from_c128(void *dst, const void *src, long long count, const double *scale,
                                double *reset_scale, cudaStream_t st)
{
    k_ff_from_c128<<<point_blocks(count), 256, 0, st>>>((float4 *)dst, (const double2 *)src, count,
                                                         scale);
    cudaError_t e = cudaGetLastError();
    // every block has read the scale once the conversion kernel is done
    if (e == cudaSuccess && reset_scale) {
        k_ff_set_one<<<1, 1, 0, st>>>(reset_scale);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_ff_from_c128_grid(void *dst, const void *src, int nx, int ny, int nz,
                                     cudaStream_t st)
{
    const int groups = (ny * nz + kFromLines - 1) / kFromLines;
    const int blocks = groups < 152 * 16 ? groups : 152 * 16;
    k_ff_from_c128_grid<<<blocks, 256, 0, st>>>((float4 *)dst, (const double2 *)src, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_observables_ff(const void *psi, const ObsArgs &a, const float2 *x2ff,
                                  const float2 *vxff, double *scratch, double *sums, cudaStream_t st)
{
    dim3 grid;
    int threads = 0;
    obs_walk_geometry(a.nx, a.ny, a.nz, grid, threads);
    k_observables_ff<<<grid, threads, 0, st>>>((const float4 *)psi, a, x2ff, vxff, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long nrows = (long long)grid.x * grid.y * grid.z;
    return launch_rows_finish(scratch, nrows, scratch + nrows * kObsWidth, sums, st);
}

cudaError_t launch_ff_to_c128(void *dst, const void *src, long long count, const double *scale,
                              cudaStream_t st)
{
    k_ff_to_c128<<<point_blocks(count), 256, 0, st>>>((double2 *)dst, (const float4 *)src, count,
                                                       scale);
    return cudaGetLastError();
}

}  // namespace gp
