// sscn_pair.cuh -- the Crank-Nicolson line update (calclux / calcluy /
// calcluz) of one line held in shared memory, solved in place by a pair of
// lanes of one warp: the tile solver of the batch engine and of the fused
// x+y slab sweep.
#pragma once

#include "sscn_accum.cuh"
#include "sscn_coef.cuh"
#include "sscn_line.cuh"

namespace gp {

// One axis' Thomas data as a pair solve reads it: the forward-elimination
// tables (m = n - 1 entries), the index from which both are constant and
// those constants, the middle-row multiplier and kappa (imaginary time: the
// real kappa; real time: kappa / i).
template <typename T> struct PairTabs {
    using F = typename Coef<T>::t;
    const F *mult, *cp;
    F minf, cinf, mid;
    int conv;
    T kappa;
};

// (I - kappa L) u = (I + kappa L) psi on row[0], row[es], ..., row[(n-1) es]
// (point 0 and the virtual point n are zero), in place, right-hand-side
// form.  The lane pair (l, l ^ 16) owns the line: the top lane (l < 16)
// eliminates i = 1 .. k-1, the bottom lane i = m .. k+1 with the mirrored
// tables (the matrix is symmetric Toeplitz), the top lane closes the middle
// row k = ceil(m / 2), and both back-substitute outward.  NL: calcnu on each
// point as the forward elimination reads it (the elimination keeps only d',
// so the updated point is never stored; the middle point is computed by
// both lanes).  norm: |u|^2 of every result into acc.  ES > 0 fixes the
// element stride at compile time, else es is used.  Every lane of the warp
// calls this (the shuffles need them all); `active` marks lanes with a line.
//
// Past the index where the tables reach their constants the recurrences run
// from registers in groups of 4 points, whose shared-memory reads (and
// calcnu) are issued before any of the group's results is stored.
template <typename T, int MODE, bool NL, int ES>
__device__ __forceinline__ void solve_pair(typename Cx<T>::t *row, int es_rt, int n, bool top,
                                           bool active, bool norm, Acc<T> &acc,
                                           const PairTabs<T> &tb, const Calcnu<T, MODE> &cu)
{
    using C = typename Cx<T>::t;
    const int es = ES > 0 ? ES : es_rt;
    const int m = n - 1;
    const int k = (m + 1) >> 1;
    const LineOps<T, MODE> cn{tb.kappa};
    const C zero = cx<T>((T)0, (T)0);
    const int len = top ? k - 1 : m - k;
    const int dir = top ? es : -es, di = top ? 1 : -1;
    const int tc = min(tb.conv, len);
    C prev = zero, cur = zero, d = zero;
    if (active) {
        C *p = row + (top ? 1 : m) * es;
        int i = top ? 1 : m;               // point index of *p
        cur = *p;
        if (NL) cur = cu.apply(cur, i);
        int t = 0;
        for (; t < tc; ++t, p += dir, i += di) {
            C next = p[dir];
            if (NL) next = cu.apply(next, i + di);
            d = cn.fwd(cn.rhs(prev, cur, next), d, tb.mult[t]);
            *p = d;
            prev = cur;
            cur = next;
        }
        for (; t + 4 <= len; t += 4, p += 4 * dir, i += 4 * di) {
            C nx[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nx[q] = p[(q + 1) * dir];
            if (NL) {
#pragma unroll
                for (int q = 0; q < 4; ++q) nx[q] = cu.apply(nx[q], i + (q + 1) * di);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d = cn.fwd(cn.rhs(prev, cur, nx[q]), d, tb.minf);
                p[q * dir] = d;
                prev = cur;
                cur = nx[q];
            }
        }
        for (; t < len; ++t, p += dir, i += di) {
            C next = p[dir];
            if (NL) next = cu.apply(next, i + di);
            d = cn.fwd(cn.rhs(prev, cur, next), d, tb.minf);
            *p = d;
            prev = cur;
            cur = next;
        }
    }
    // top: prev = psi_{k-1}, cur = psi_k; bottom: prev = psi_{k+1}, d = e_{k+1}
    const C o_prev = cx<T>(__shfl_xor_sync(0xffffffffu, prev.x, 16), __shfl_xor_sync(0xffffffffu, prev.y, 16));
    const C o_d = cx<T>(__shfl_xor_sync(0xffffffffu, d.x, 16), __shfl_xor_sync(0xffffffffu, d.y, 16));
    C vk = zero;
    if (active && top) {
        vk = cn.fwd(cn.rhs(prev, cur, o_prev), cx<T>(d.x + o_d.x, d.y + o_d.y), tb.mid);
        row[k * es] = vk;
        if (norm) acc.add(fma(vk.x, vk.x, vk.y * vk.y));
    }
    const C o_vk = cx<T>(__shfl_xor_sync(0xffffffffu, vk.x, 16), __shfl_xor_sync(0xffffffffu, vk.y, 16));
    C u = top ? vk : o_vk;
    if (active) {
        int t = len - 1;
        C *p = row + (top ? 1 + t : m - t) * es;
        for (; t - 3 >= tc; t -= 4, p -= 4 * dir) {
            C dv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) dv[q] = p[-q * dir];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                u = cn.back(dv[q], tb.cinf, u);
                p[-q * dir] = u;
                if (norm) acc.add(fma(u.x, u.x, u.y * u.y));
            }
        }
        for (; t >= tc; --t, p -= dir) {
            u = cn.back(*p, tb.cinf, u);
            *p = u;
            if (norm) acc.add(fma(u.x, u.x, u.y * u.y));
        }
        for (; t >= 0; --t, p -= dir) {
            u = cn.back(*p, tb.cp[t], u);
            *p = u;
            if (norm) acc.add(fma(u.x, u.x, u.y * u.y));
        }
    }
}

}  // namespace gp
