// sscn_seg.cuh -- the Crank-Nicolson line update (calclux / calcluy /
// calcluz) of one line held in shared memory, split into S segments solved
// at once by S lanes of one warp: the batch engine's solver for its longer
// lines.
//
// The elimination coefficients of a constant-coefficient line converge
// geometrically (|c'_i| -> |c'_inf| < 1), so the forward elimination over a
// segment can start W points before it from d' = 0 and the back substitution
// W points after it from u = 0: the dropped start values reach the segment
// damped by |c'|^W.  The host picks W so that max|c'|^(W+1) lies below the
// storage precision's rounding (a window that reaches the end of the line
// starts exactly there).  Each lane then runs about m / S + W steps in each
// direction where the two-ended pair solve runs m / 2.
#pragma once

#include <type_traits>

#include "sscn_accum.cuh"
#include "sscn_coef.cuh"
#include "sscn_line.cuh"
#include "sscn_pair.cuh"

namespace gp {

// First point of segment s of the interior points 1 .. m: the nearly equal
// split, moved up by one where needed so that segment starts alternate odd,
// even, odd, ...  In a column-major tile (point c of line r at c R + r) and
// in a row-major tile whose pitch is 2 mod 4, lanes of segments of opposite
// parity then fall in disjoint halves of the shared-memory banks.
template <int S> __device__ __forceinline__ int seg_start(int s, int m)
{
    int a = 1 + (s * m) / S;
    if ((a ^ (s + 1)) & 1) ++a;
    return a;
}

// (I - kappa L) u = (I + kappa L) psi on row[0], row[es], ..., row[(n-1) es]
// (point 0 and the virtual point n are zero), in place, right-hand-side
// form, by S lanes: lane `seg` owns points a .. b.  Four phases separated by
// warp barriers, so that no lane reads a point another lane has already
// overwritten:
//   A  forward over the look-back window max(1, a - W) .. a - 1 (reads only);
//   B  forward over a .. b, d' in place (the point b + 1, the next segment's
//      first, was read in phase A);
//   C  back substitution over min(m, b + W) .. b + 1 from u = 0 (reads d' only);
//   D  back substitution over b .. a, u in place.
// NL: calcnu on each point as the forward elimination reads it (window
// points too, so a point's calcnu may be computed by two lanes, identically).
// norm: |u|^2 of every result into acc.  Every lane of the warp calls this
// (the barriers need them all); `active` marks lanes with a line.
//
// The tables hold the exact coefficients (m entries, 0-based: point i uses
// entry i - 1); from index conv on they equal the constants minf / cinf,
// which the recurrences then take from registers in groups of 4 points
// whose shared-memory reads (and calcnu) are issued before any result of
// the group is stored.
template <typename T, int MODE, bool NL, int ES, int S>
__device__ __forceinline__ void solve_seg(typename Cx<T>::t *row, int es_rt, int n, int seg, int W,
                                          bool active, bool norm, Acc<T> &acc, const PairTabs<T> &tb,
                                          const Calcnu<T, MODE> &cu)
{
    using C = typename Cx<T>::t;
    const int es = ES > 0 ? ES : es_rt;
    const int m = n - 1;
    const LineOps<T, MODE> cn{tb.kappa};
    const C zero = cx<T>((T)0, (T)0);
    const int a = seg_start<S>(seg, m);
    const int b = seg == S - 1 ? m : seg_start<S>(seg + 1, m) - 1;
    auto ld = [&](int i) {
        C v = row[i * es];
        if (NL) v = cu.apply(v, i);
        return v;
    };
    // forward elimination over points i .. ie - 1, reading psi up to point ie
    auto fwd_span = [&](auto store, int i, int ie, C &prev, C &cur, C &d) {
        constexpr bool ST = decltype(store)::value;
        for (; i < ie && i - 1 < tb.conv; ++i) {
            const C next = ld(i + 1);
            d = cn.fwd(cn.rhs(prev, cur, next), d, tb.mult[i - 1]);
            if (ST) row[i * es] = d;
            prev = cur;
            cur = next;
        }
        for (; i + 4 <= ie; i += 4) {
            C nx[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nx[q] = row[(i + 1 + q) * es];
            if (NL) {
#pragma unroll
                for (int q = 0; q < 4; ++q) nx[q] = cu.apply(nx[q], i + 1 + q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d = cn.fwd(cn.rhs(prev, cur, nx[q]), d, tb.minf);
                if (ST) row[(i + q) * es] = d;
                prev = cur;
                cur = nx[q];
            }
        }
        for (; i < ie; ++i) {
            const C next = ld(i + 1);
            d = cn.fwd(cn.rhs(prev, cur, next), d, tb.minf);
            if (ST) row[i * es] = d;
            prev = cur;
            cur = next;
        }
    };
    // back substitution over points i, i - 1, .. ie (i >= ie - 1)
    auto bwd_span = [&](auto store, int i, int ie, C &u) {
        constexpr bool ST = decltype(store)::value;
        for (; i - 3 >= ie && i - 4 >= tb.conv; i -= 4) {
            C dv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) dv[q] = row[(i - q) * es];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u = cn.back(dv[q], tb.cinf, u);
                if (ST) {
                    row[(i - q) * es] = u;
                    if (norm) acc.add(fma(u.x, u.x, u.y * u.y));
                }
            }
        }
        for (; i >= ie; --i) {
            u = cn.back(row[i * es], i - 1 >= tb.conv ? tb.cinf : tb.cp[i - 1], u);
            if (ST) {
                row[i * es] = u;
                if (norm) acc.add(fma(u.x, u.x, u.y * u.y));
            }
        }
    };
    using yes = std::true_type;
    using no = std::false_type;
    // A: the look-back window; d' = 0 before its first point (exact at 1)
    C prev = zero, cur = zero, d = zero, right = zero;
    if (active) {
        const int i0 = max(1, a - W);
        prev = i0 > 1 ? ld(i0 - 1) : zero;
        cur = ld(i0);
        fwd_span(no{}, i0, a, prev, cur, d);
        right = b < m ? ld(b + 1) : zero;
    }
    __syncwarp();
    // B: the segment, d' in place
    if (active) {
        fwd_span(yes{}, a, b, prev, cur, d);
        d = cn.fwd(cn.rhs(prev, cur, right), d, b - 1 < tb.conv ? tb.mult[b - 1] : tb.minf);
        row[b * es] = d;
    }
    __syncwarp();
    // C: u at point b + 1 from the look-ahead window; u = 0 after its last
    // point (exact at m)
    C u = zero;
    if (active && b < m) bwd_span(no{}, min(m, b + W), b + 1, u);
    __syncwarp();
    // D: the segment, u in place
    if (active) bwd_span(yes{}, b, a, u);
}

}  // namespace gp
