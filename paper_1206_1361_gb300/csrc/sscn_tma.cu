// sscn_tma.cu -- TMA-pipelined Crank-Nicolson sweeps (calclux / calcluy /
// calcluz, with calcnu fused into the x sweep) for the bandwidth-bound
// complex64 form, sm_103a.
//
// One CTA owns a tile of L = 32 K lines (one consumer thread per line) and
// walks them chunk by chunk: a chunk is the C consecutive points of all L
// lines, one TMA box.  A producer warp keeps up to S - 1 chunks in flight
// ahead of the compute through an S-stage shared-memory ring
// (cp.async.bulk.tensor loads completing on one mbarrier per stage); ragged
// tiles and the points past the end of a line arrive as zeros (TMA
// out-of-bounds fill) and are clipped on the way back.
//
// Each consumer thread runs the forward elimination of its line through the
// tile, keeping d'_i for the last two chunks in a shared-memory ring, and
// writes the finished values back into the tile in place; the producer then
// stores the tile with a TMA store and reuses the stage.  The complex64 path
// eliminates in increment form, (I - kappa L) D = kappa L psi, u = psi + 2 D,
// so that only the final store rounds at full size: repeated every step on a
// smooth state, the FP32 roundings of u = 2 v - psi do not average out and
// the real-time norm drifts.  Its forward pass runs one point behind the
// newest loaded point, which supplies psi_{i+1}.  Back substitution is windowed: the values of chunk q-1
// are produced after the forward pass of chunk q, starting from v ~ d' at the
// end of chunk q.  The dropped term is c'_e v_{e+1}, damped by |c'| at every
// step back; the seed sits W points into chunk q, so every output carries an
// error below |c'|^(W+1) max|v|.  The host picks the smallest W <= C for which
// that bound is under 2^-40 (complex64) / 2^-55 (complex128) -- far below one
// rounding, because the truncation is the same linear perturbation at every
// step -- and otherwise uses the exact one-line-per-thread kernel.
// The last two chunks are back-substituted exactly from v_m = d'_m.
//
// Layout of a stage: x sweep -> [L rows][C points] with the 128-byte TMA
// swizzle (16-byte chunk j of row r sits at j ^ (r % 8)), so a warp reading
// point c of 32 different rows hits distinct banks; y / z sweeps ->
// [C rows][L points], consecutive threads on consecutive addresses.

#include <cstdint>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "sscn_accum.cuh"
#include "sscn_internal.h"
#include "sscn_line.cuh"
#include "sscn_tma.cuh"

#ifndef GP_TMA_HI_ONLY
#define GP_TMA_HI_ONLY 1
#endif

namespace gp {
namespace {

using namespace gp::tma;

template <typename T> struct CT2;
template <> struct CT2<double> { using c = double2; };
template <> struct CT2<float> { using c = float2; };

template <typename T> __device__ __forceinline__ typename CT2<T>::c mk2(T x, T y)
{
    typename CT2<T>::c r;
    r.x = x;
    r.y = y;
    return r;
}

// ------------------------------------------------------------------ kernel

struct TmaArgs {
    int n;              // stored points per line (m = n - 1 unknowns)
    int lines_a;        // extent of the in-tile line index (y for x, x for y / z)
    int win;            // look-back window W (1 .. C)
    int conv;           // table index from which c' and mult are constant
    double2 cinf64, minf64;     // those constants, FP64 path
    float4 cinf32, minf32;      // those constants, complex64 path (hi + lo)
    const void *cp, *mult;      // coefficient tables (Coef<T>), m entries
    const void *px, *py, *pz;   // calcnu factor tables (x sweep)
    const float *tx, *ty, *tz;  // complex64 phase tables (x sweep)
    double kappa;       // kre (imaginary time) or kim (real time)
    StepG g;            // G of the fused pointwise step
    const double *scale;
    double *partials;   // norm partials (NORM)
    int *err;           // device error bits
};

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per chunk wait
constexpr int kErrTimeout = 2;
// Columns of tensor memory a CTA of the TMEM-ring shapes allocates: d' of
// two chunks, 32 FP32 words per chunk (16 complex64 points).
constexpr int kTmemCols = 64;

template <typename T, int L, int C, int S, int AXIS>
struct TileGeom {
    static constexpr int E = (int)sizeof(typename CT2<T>::c);   // bytes per complex value
    static constexpr int U = E / 8;                              // 8-byte TMA units per value
    static constexpr int kStageBytes = L * C * E;
    // byte offset of (line l, point c) inside a stage
    static __device__ __forceinline__ int off(int l, int c)
    {
        if (AXIS == 0) {
            const int byte = c * E;                 // within the 128-byte row of line l
            return l * (C * E) + ((((byte >> 4) ^ (l & 7))) << 4) + (byte & 15);
        }
        return (c * L + l) * E;
    }
};

// Warp-specialised CTA: K consumer warps own L = 32 K lines (one per
// thread); warp K is the producer, whose lane 0 issues every TMA load and
// store.  Per stage s: full[s] completes when a chunk's bytes have landed,
// ready[s] when all K consumer warps have written the chunk's final values
// (one arrival per warp).  The producer stores a chunk once it is ready and
// reuses its stage only after that store has read shared memory, so the
// consumers never wait on a store.
// NL: calcnu on each point as it arrives (x sweep); NLOUT: calcnu on each
// result before it is stored (the symmetric splitting's second half step in
// the last real-time sweep).
// TM (complex64): the d' ring lives in tensor memory, each consumer thread's
// line in its TMEM lane, which leaves shared memory to the stages and admits
// more resident CTAs; every lane of a consumer warp then runs the same
// instruction stream (the tcgen05 accesses are warp-wide), lanes past the end
// of a ragged tile computing on the zeros TMA filled in, whose rows the TMA
// store clips.
template <typename T, int K, int C, int S, bool TM>
constexpr size_t tma_smem_bytes()
{
    constexpr size_t L = 32 * K;
    return 1024 + (size_t)S * L * C * sizeof(typename CT2<T>::c) +
           (TM ? 0 : 2 * (size_t)C * L * sizeof(typename CT2<T>::c)) + 2 * S * sizeof(uint64_t) +
           32 * sizeof(double) + 16;
}

// Resident CTAs per SM the TMEM shapes are built for: as many as shared
// memory admits, at most 512 / kTmemCols.
template <typename T, int K, int C, int S, bool TM>
constexpr int tma_min_blocks()
{
    if (!TM) return 1;
    constexpr int by_smem = (int)((227 * 1024) / tma_smem_bytes<T, K, C, S, TM>());
    constexpr int by_tmem = 512 / kTmemCols;
    return by_smem < by_tmem ? by_smem : by_tmem;
}

template <typename T, int MODE, int AXIS, bool NL, bool NORM, int K, int C, int S, bool TM,
          bool NLOUT = false>
__global__ void __launch_bounds__(32 * (K + 1), (tma_min_blocks<T, K, C, S, TM>()))
k_sweep_tma(const __grid_constant__ CUtensorMap map, const TmaArgs args)
{
    static_assert(!TM || (sizeof(T) == 4 && C == 16), "the TMEM ring holds complex64 chunks of 16");
    using Cv = typename CT2<T>::c;
    constexpr int L = 32 * K;
    using G = TileGeom<T, L, C, S, AXIS>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the stage ring (the 128-byte swizzle needs it)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *stages = smem;
    Cv *ring = reinterpret_cast<Cv *>(stages + S * G::kStageBytes);     // [2][C][L]
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (TM ? 0 : 2 * C * L));
    uint64_t *ready = full + S;
    double *red = reinterpret_cast<double *>(ready + S);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(red + 32);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == K;
    const int l = producer ? 0 : threadIdx.x;        // line inside the tile
    const int tile0 = blockIdx.x * L;
    const int a = tile0 + l;
    const bool active = !producer && a < args.lines_a;
    const bool run = TM ? !producer : active;       // computes (see TM above)
    const int m = args.n - 1;
    const int Q = (args.n + C - 1) / C;             // chunks covering stored points 0 .. m
    using F = typename Coef<T>::t;
    const F *cp_tab = static_cast<const F *>(args.cp);
    const F *mult_tab = static_cast<const F *>(args.mult);
    // complex64 eliminates in increment form (below), where the rounding of
    // the coefficients enters scaled by the small kappa L psi, so the hi
    // parts suffice
    constexpr bool INC = sizeof(T) == 4;
    constexpr bool HI = INC && GP_TMA_HI_ONLY;
    const LineOps<T, MODE, HI> cn{(T)args.kappa};
    const int conv = args.conv, win = args.win;
    F cinf, minf;
    if constexpr (sizeof(T) == 8) {
        cinf = args.cinf64;
        minf = args.minf64;
    } else {
        cinf = args.cinf32;
        minf = args.minf32;
    }
    // table entry t (0-based): past `conv` every entry equals the last one
    auto cp = [&](int t) { return t < conv ? cp_tab[t] : cinf; };
    auto mult = [&](int t) { return t < conv ? mult_tab[t] : minf; };

    // TMA coordinates (innermost first, in 8-byte units) of chunk q
    auto coords = [&](int q, int &c0, int &c1, int &c2) {
        if (AXIS == 0) { c0 = q * C * G::U; c1 = tile0; c2 = blockIdx.y; }
        else if (AXIS == 1) { c0 = tile0 * G::U; c1 = q * C; c2 = blockIdx.y; }
        else { c0 = tile0 * G::U; c1 = blockIdx.y; c2 = q * C; }
    };
    auto stage_ptr = [&](int q) { return stages + (q % S) * G::kStageBytes; };
    auto at = [&](int q, int c) -> Cv * { return reinterpret_cast<Cv *>(stage_ptr(q) + G::off(l, c)); };

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
    Acc<T> nacc;
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
                    // the stage last held chunk q - S: store it once final,
                    // then let the store finish reading before reloading
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
        Calcnu<T, MODE> nl{};
        if ((NL || NLOUT) && run) {
            // lanes past a ragged tile's end take the last line's factors
            const F *py = static_cast<const F *>(args.py), *pz = static_cast<const F *>(args.pz);
            nl.setup(static_cast<const F *>(args.px), py, pz, args.tx, args.ty, args.tz,
                     active ? a : args.lines_a - 1, blockIdx.y, args.g.value(), args.scale);
        }
        // complex64: increment form with the forward pass one point behind
        // the newest point (it needs psi_{i+1}); FP64: u = 2 v - psi
        auto slot = [&](int i) -> Cv & { return ring[((i / C) & 1) * C * L + (i % C) * L + l]; };
        // TMEM column of point i: chunk parity, then 2 words per point
        auto tcol = [&](int i) -> uint32_t { return (uint32_t)((((i / C) & 1) * C + i % C) * 2); };
        auto put = [&](int i, Cv d) {
            if constexpr (TM) tmem_st2(tbase + tcol(i), d.x, d.y);
            else slot(i) = d;
        };
        auto get = [&](int i) -> Cv {
            if constexpr (TM) {
                const float2 v = tmem_ld2(tbase + tcol(i));
                return mk2<T>(v.x, v.y);
            } else {
                return slot(i);
            }
        };
        auto output = [&](Cv v, Cv *tile_slot, int i) {
            Cv u = INC ? LineOps<T, MODE>::out_inc(v, *tile_slot) : LineOps<T, MODE>::out(v, *tile_slot);
            if (NLOUT) u = nl.apply(u, i);
            *tile_slot = u;
            if (NORM && active) nacc.add(fma(u.x, u.x, u.y * u.y));
        };
        const Cv zero = mk2<T>((T)0, (T)0);
        Cv d = zero, pa = zero, pb = zero;          // INC: psi~_{i-1}, psi~_i
        for (int q = 0; q < Q; ++q) {
            bool ok = mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kWaitLimitNs);
            if (TM) ok = __all_sync(0xffffffffu, ok);    // the warp leaves together
            if (!ok) {
                failed = true;
                break;
            }
            const bool last = q == Q - 1;
            // Interior chunks -- all points unknowns, tables converged to their
            // constants, neither the first chunks nor the last -- take a path
            // with no guards, no table loads and compile-time offsets.
            const bool fast = run && q >= 2 && !last && (q - 1) * C - 1 >= conv &&
                              (q + 1) * C - 1 <= m;
            if (fast) {
                unsigned char *sq = stage_ptr(q), *sp = stage_ptr(q - 1);
                Cv *rq = ring + (q & 1) * C * L + l, *rp = ring + ((q - 1) & 1) * C * L + l;
                // one forward step at point c of chunk q
                auto fwd_at = [&](int c, Cv pj) {
                    if (INC) {
                        d = cn.fwd(cn.lap(pa, pb, pj), d, minf);
                        if constexpr (TM) put(q * C + c - 1, d);
                        else if (c == 0) rp[(C - 1) * L] = d;
                        else rq[(c - 1) * L] = d;
                        pa = pb;
                        pb = pj;
                    } else {
                        d = cn.fwd(pj, d, minf);
                        rq[c * L] = d;
                    }
                };
                // the updated value at point c of chunk q - 1 from v and psi there
                auto final_at = [&](Cv v, Cv p, int c) {
                    Cv u = INC ? LineOps<T, MODE>::out_inc(v, p) : LineOps<T, MODE>::out(v, p);
                    if (NLOUT) u = nl.apply(u, (q - 1) * C + c);
                    if (NORM && active) nacc.add(fma(u.x, u.x, u.y * u.y));
                    return u;
                };
                if constexpr (AXIS == 0 && sizeof(T) == 4) {
                    // x tiles of complex64: a swizzled 16-byte chunk holds points
                    // (c, c + 1) of a line; moving both in one access keeps the
                    // warp's 32 rows on distinct banks
                    // (unrolled by 4 pairs, not 8: the fully unrolled loop with
                    // calcnu ran 4 % slower, its code stalling the instruction fetch)
#pragma unroll 4
                    for (int c = 0; c < C; c += 2) {
                        float4 *t2 = reinterpret_cast<float4 *>(sq + G::off(l, c));
                        const float4 w = *t2;
                        Cv p0 = mk2<T>(w.x, w.y), p1 = mk2<T>(w.z, w.w);
                        if (NL) {
                            p0 = nl.apply(p0, q * C + c);
                            p1 = nl.apply(p1, q * C + c + 1);
                            *t2 = make_float4(p0.x, p0.y, p1.x, p1.y);
                        }
                        fwd_at(c, p0);
                        fwd_at(c + 1, p1);
                    }
                    if constexpr (TM) {
                        // window: the seed d'_{W-1} by its own load (a runtime
                        // column), back through points W-2 .. 0 of chunk q,
                        // then chunk q - 1 loaded whole
                        Cv v = get(q * C + win - 1);
                        {
                            float r[32];
                            tmem_ld32(tbase + tcol(q * C), r);
#pragma unroll
                            for (int c = C - 2; c >= 0; --c)
                                if (c <= win - 2) v = cn.back(mk2<T>(r[2 * c], r[2 * c + 1]), cinf, v);
                        }
                        float r[32];
                        tmem_ld32(tbase + tcol((q - 1) * C), r);
#pragma unroll
                        for (int c = C - 1; c >= 1; c -= 2) {
                            float4 *t2 = reinterpret_cast<float4 *>(sp + G::off(l, c - 1));
                            const float4 w = *t2;
                            v = cn.back(mk2<T>(r[2 * c], r[2 * c + 1]), cinf, v);
                            const Cv u1 = final_at(v, mk2<T>(w.z, w.w), c);
                            v = cn.back(mk2<T>(r[2 * c - 2], r[2 * c - 1]), cinf, v);
                            const Cv u0 = final_at(v, mk2<T>(w.x, w.y), c - 1);
                            *t2 = make_float4(u0.x, u0.y, u1.x, u1.y);
                        }
                    } else {
                    Cv v = rq[(win - 1) * L];
                    for (int c = win - 2; c >= 0; --c) v = cn.back(rq[c * L], cinf, v);
#pragma unroll
                    for (int c = C - 1; c >= 1; c -= 2) {
                        float4 *t2 = reinterpret_cast<float4 *>(sp + G::off(l, c - 1));
                        const float4 w = *t2;
                        v = cn.back(rp[c * L], cinf, v);
                        const Cv u1 = final_at(v, mk2<T>(w.z, w.w), c);
                        v = cn.back(rp[(c - 1) * L], cinf, v);
                        const Cv u0 = final_at(v, mk2<T>(w.x, w.y), c - 1);
                        *t2 = make_float4(u0.x, u0.y, u1.x, u1.y);
                    }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        Cv *tc = reinterpret_cast<Cv *>(sq + G::off(l, c));
                        Cv pj = *tc;
                        if (NL) {
                            pj = nl.apply(pj, q * C + c);
                            *tc = pj;
                        }
                        fwd_at(c, pj);
                    }
                    if constexpr (TM) {
                        Cv v = get(q * C + win - 1);
                        {
                            float r[32];
                            tmem_ld32(tbase + tcol(q * C), r);
#pragma unroll
                            for (int c = C - 2; c >= 0; --c)
                                if (c <= win - 2) v = cn.back(mk2<T>(r[2 * c], r[2 * c + 1]), cinf, v);
                        }
                        float r[32];
                        tmem_ld32(tbase + tcol((q - 1) * C), r);
#pragma unroll
                        for (int c = C - 1; c >= 0; --c) {
                            Cv *tc = reinterpret_cast<Cv *>(sp + G::off(l, c));
                            v = cn.back(mk2<T>(r[2 * c], r[2 * c + 1]), cinf, v);
                            *tc = final_at(v, *tc, c);
                        }
                    } else {
                    Cv v = rq[(win - 1) * L];
                    for (int c = win - 2; c >= 0; --c) v = cn.back(rq[c * L], cinf, v);
#pragma unroll
                    for (int c = C - 1; c >= 0; --c) {
                        Cv *tc = reinterpret_cast<Cv *>(sp + G::off(l, c));
                        v = cn.back(rp[c * L], cinf, v);
                        *tc = final_at(v, *tc, c);
                    }
                    }
                }
            } else {
                // forward elimination through chunk q
                if (run) {
#pragma unroll 4
                    for (int c = 0; c < C; ++c) {
                        const int j = q * C + c;
                        if (INC) {
                            Cv pj = zero;
                            if (j <= m) {
                                pj = *at(q, c);
                                if (NL && j >= 1) {
                                    pj = nl.apply(pj, j);
                                    *at(q, c) = pj;
                                }
                            }
                            const int i = j - 1;
                            if (i >= 1 && i <= m) {
                                d = cn.fwd(cn.lap(pa, pb, pj), d, mult(i - 1));
                                put(i, d);
                            }
                            pa = pb;
                            pb = pj;
                        } else if (j >= 1 && j <= m) {
                            Cv p = *at(q, c);
                            if (NL) {
                                p = nl.apply(p, j);
                                *at(q, c) = p;
                            }
                            d = cn.fwd(p, d, mult(j - 1));
                            put(j, d);
                        }
                    }
                    if (INC && last && Q * C - 1 == m) {
                        // point m: its right neighbour is the virtual zero node
                        d = cn.fwd(cn.lap(pa, pb, zero), d, mult(m - 1));
                        put(m, d);
                    }
                }
                if (run) {
                    if (!last && q >= 1) {
                        // windowed: seed W points into chunk q, output chunk q - 1
                        Cv v = get(q * C + win - 1);
                        for (int c = win - 2; c >= 0; --c)
                            v = cn.back(get(q * C + c), cp(q * C + c - 1), v);
#pragma unroll 4
                        for (int c = C - 1; c >= 0; --c) {
                            const int i = (q - 1) * C + c;
                            if (i < 1) break;
                            v = cn.back(get(i), cp(i - 1), v);
                            output(v, at(q - 1, c), i);
                        }
                    } else if (last) {
                        // exact: v_m = d'_m, down through chunks q and q - 1
                        Cv v = d;
                        const int lo = q >= 1 ? (q - 1) * C : 0;
                        for (int i = m; i >= lo && i >= 1; --i) {
                            if (i < m) v = cn.back(get(i), cp(i - 1), v);
                            output(v, at(i / C, i % C), i);
                        }
                    }
                }
            }
            if (q >= 1 || last) {
                fence_proxy_async();             // tile writes -> async proxy
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
        // block sum of the per-line norm contributions, fixed order
        double v = nacc.get();
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

template <typename T, int MODE, int AXIS, bool NL, bool NORM, int K, int C, int S, bool TM,
          bool NLOUT = false>
cudaError_t launch_tma_inst(const CUtensorMap &map, const TmaArgs &args, int tiles, int lines_b,
                            cudaStream_t st)
{
    auto kern = k_sweep_tma<T, MODE, AXIS, NL, NORM, K, C, S, TM, NLOUT>;
    constexpr int threads = 32 * (K + 1);
    static size_t smem_of[64] = {};           // per device ordinal, 0: not configured
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!smem_of[dev]) {
        size_t smem = tma_smem_bytes<T, K, C, S, TM>();
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
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, threads, smem);
            if (e != cudaSuccess) return e;
            if (blocks * kTmemCols <= 512) break;
            smem += 1024;
            if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        }
        smem_of[dev] = smem;
    }
    kern<<<dim3(tiles, lines_b), threads, smem_of[dev], st>>>(map, args);
    return cudaGetLastError();
}

template <typename T, int AXIS, int K, int C, int S, bool TM>
cudaError_t launch_tma_axis(int mode, bool nl, bool norm, bool nlout, const CUtensorMap &map,
                            const TmaArgs &args, int tiles, int lines_b, cudaStream_t st)
{
    // the symmetric splitting's second half step: real time, y or z sweep
    if (nlout) {
        if constexpr (AXIS == 0) return cudaErrorInvalidValue;
        else {
            if (mode != 1 || norm || nl) return cudaErrorInvalidValue;
            return launch_tma_inst<T, 1, AXIS, false, false, K, C, S, TM, true>(map, args, tiles,
                                                                               lines_b, st);
        }
    }
    // calcnu is fused into the x sweep only
#define GP_TMA(MODE, NLV, NORMV)                                                             \
    return launch_tma_inst<T, MODE, AXIS, (NLV && AXIS == 0), NORMV, K, C, S, TM>(map, args,   \
                                                                               tiles, lines_b, st)
    if (mode == 0) {
        if (nl) { if (norm) GP_TMA(0, true, true); GP_TMA(0, true, false); }
        if (norm) GP_TMA(0, false, true);
        GP_TMA(0, false, false);
    }
    if (nl) { if (norm) GP_TMA(1, true, true); GP_TMA(1, true, false); }
    if (norm) GP_TMA(1, false, true);
    GP_TMA(1, false, false);
#undef GP_TMA
}

// Tile shapes (consumer warps K, points per chunk C, stages S); a CTA owns
// 32 K lines.  C is fixed by the 128-byte swizzled x rows (16 complex64 / 8
// complex128 points); K and S trade CTAs per SM against chunks in flight.
// TM: the d' ring in tensor memory (complex64 only).
struct Shape { int K, C, S; bool TM; };
// Index 0 is the default: the fastest measured at 512 x 512 x 256 complex64
// (4 consumer warps, 3 stages, TMEM ring: 16 consumer warps per SM against
// 10 with the ring in shared memory) and 256^3 complex128.
constexpr Shape kShapes32[] = {{4, 16, 3, true},  {2, 16, 3, true},  {2, 16, 4, true},
                               {2, 16, 3, false}, {1, 16, 4, false}, {2, 16, 4, false},
                               {4, 16, 3, false}, {1, 16, 3, false}};
constexpr Shape kShapes64[] = {{1, 8, 4, false}, {2, 8, 4, false}, {4, 8, 3, false}};
constexpr int kNumShapes32 = 8, kNumShapes64 = 3;

template <typename T, int K, int C, int S, bool TM>
cudaError_t launch_shape(int mode, int axis, bool nl, bool norm, bool nlout, const CUtensorMap &map,
                         const TmaArgs &args, int tiles, int lines_b, cudaStream_t st)
{
    if (axis == 0) return launch_tma_axis<T, 0, K, C, S, TM>(mode, nl, norm, nlout, map, args, tiles, lines_b, st);
    if (axis == 1) return launch_tma_axis<T, 1, K, C, S, TM>(mode, nl, norm, nlout, map, args, tiles, lines_b, st);
    return launch_tma_axis<T, 2, K, C, S, TM>(mode, nl, norm, nlout, map, args, tiles, lines_b, st);
}

Shape shape_of(int prec, int shape)
{
    if (prec == kC128) return kShapes64[shape < 0 || shape >= kNumShapes64 ? 0 : shape];
    return kShapes32[shape < 0 || shape >= kNumShapes32 ? 0 : shape];
}

}  // namespace

int tma_shapes(int prec) { return prec == kC128 ? kNumShapes64 : kNumShapes32; }
int tma_chunk(int prec, int shape) { return shape_of(prec, shape).C; }
int tma_lines(int prec, int shape) { return 32 * shape_of(prec, shape).K; }

int tma_blocks(int prec, int shape, const SweepGeom &g)
{
    const int L = tma_lines(prec, shape);
    return ((g.lines_a + L - 1) / L) * g.lines_b;
}

// Encode the tensor map of psi for one sweep axis.  psi is viewed as a 3D
// array of 8-byte units {U * nx, ny, nz}; the box is one chunk of one tile.
cudaError_t make_sweep_map(int prec, int shape, void *psi, int nx, int ny, int nz, int axis,
                           CUtensorMap *out)
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
    const int U = prec == kC128 ? 2 : 1;
    const Shape sh = shape_of(prec, shape);
    const cuuint64_t dims[3] = {(cuuint64_t)U * nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)U * nx * 8, (cuuint64_t)U * nx * ny * 8};
    cuuint32_t box[3];
    CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    const int L = 32 * sh.K;
    if (axis == 0) { box[0] = U * sh.C; box[1] = L; box[2] = 1; sw = CU_TENSOR_MAP_SWIZZLE_128B; }
    else if (axis == 1) { box[0] = U * L; box[1] = sh.C; box[2] = 1; }
    else { box[0] = U * L; box[1] = 1; box[2] = sh.C; }
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, psi, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma(int prec, int shape, int mode, int axis, const CUtensorMap &map,
                             const AxisTables &ax, const SweepGeom &g, const NonlinArgs *nl,
                             const Partials *norm_out, int *err, cudaStream_t st, bool nl_at_output)
{
    TmaArgs args{};
    args.n = g.n;
    args.lines_a = g.lines_a;
    args.kappa = mode == 0 ? ax.kre : ax.kim;
    args.partials = norm_out ? norm_out->buf : nullptr;
    args.err = err;
    if (prec == kC128) {
        args.cp = ax.cp64;
        args.mult = ax.mult64;
        args.conv = ax.conv64;
        args.win = ax.win64;
        args.cinf64 = ax.cinf64;
        args.minf64 = ax.minf64;
    } else {
        args.cp = ax.cp32;
        args.mult = ax.mult32;
        args.conv = ax.conv32;
        args.win = ax.win32;
        args.cinf32 = ax.cinf32;
        args.minf32 = ax.minf32;
    }
    if (nl) {
        args.px = prec == kC128 ? (const void *)nl->px : (const void *)nl->px32;
        args.py = prec == kC128 ? (const void *)nl->py : (const void *)nl->py32;
        args.pz = prec == kC128 ? (const void *)nl->pz : (const void *)nl->pz32;
        args.tx = nl->tx32;
        args.ty = nl->ty32;
        args.tz = nl->tz32;
        args.g = nl->g;
        args.scale = nl->scale;
    }
    const int tiles = (g.lines_a + tma_lines(prec, shape) - 1) / tma_lines(prec, shape);
    const bool norm = norm_out != nullptr, has_nl = nl != nullptr && !nl_at_output;
    const bool nlout = nl != nullptr && nl_at_output;
    const int lb = g.lines_b;
#define GP_SHAPE(T, SH, I)                                                                   \
    if (shape == I)                                                                          \
        return launch_shape<T, SH[I].K, SH[I].C, SH[I].S, SH[I].TM>(mode, axis, has_nl, norm,   \
                                                                    nlout, map, args, tiles, lb, st)
    if (prec == kC128) {
        GP_SHAPE(double, kShapes64, 1);
        GP_SHAPE(double, kShapes64, 2);
        GP_SHAPE(double, kShapes64, 0);
        return cudaErrorInvalidValue;
    }
    GP_SHAPE(float, kShapes32, 1);
    GP_SHAPE(float, kShapes32, 2);
    GP_SHAPE(float, kShapes32, 3);
    GP_SHAPE(float, kShapes32, 4);
    GP_SHAPE(float, kShapes32, 5);
    GP_SHAPE(float, kShapes32, 6);
    GP_SHAPE(float, kShapes32, 7);
    GP_SHAPE(float, kShapes32, 0);
#undef GP_SHAPE
    return cudaErrorInvalidValue;
}

}  // namespace gp
