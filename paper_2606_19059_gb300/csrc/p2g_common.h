// p2g_common.h -- pieces shared by the owner-computes P2G kernels (eq. (p2g)):
// the per-tile table of neighbour-tile point ranges and the lookup of one
// candidate in their concatenation.
#pragma once

#include <stdint.h>

namespace ewg {

constexpr int kP2GThreads = 256;
constexpr int kP2GCandidates = 2;  // candidates per thread and round (512 a round)
constexpr int kP2GMaxSeg = 125;    // (KT+1)^3 with KT <= 4 (T = 4, P = 16)

__device__ __forceinline__ int p2g_wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Warp 0 of the block writes the segment table of tile (tx, ty, tz): segment
// s = (dz, dy, dx) in [-KT, 0]^3 (x fastest) is the point range of the
// periodic neighbour tile at that offset, seg_start[s] its first point and
// seg_pref[s] the number of points in the segments before it.  The caller
// synchronises the block before reading the table.
__device__ __forceinline__ void p2g_segment_table(const int32_t *startt, int nt, int KT, int tx, int ty, int tz,
                                                  int *seg_start, int *seg_pref)
{
    if (threadIdx.x >= 32)
        return;
    const int side = KT + 1, nseg = side * side * side;
    int carry = 0;
    for (int s0 = 0; s0 < nseg; s0 += 32) {
        const int s = s0 + threadIdx.x;
        int len = 0;
        if (s < nseg) {
            const int dx = s % side - KT, dy = (s / side) % side - KT, dz = s / (side * side) - KT;
            const int nb = (p2g_wrapi(tz + dz, nt) * nt + p2g_wrapi(ty + dy, nt)) * nt + p2g_wrapi(tx + dx, nt);
            seg_start[s] = startt[nb];
            len = startt[nb + 1] - startt[nb];
        }
        int v = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)threadIdx.x >= o)
                v += u;
        }
        if (s < nseg)
            seg_pref[s + 1] = carry + v;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (threadIdx.x == 0)
        seg_pref[0] = 0;
}

// Candidate q (0 <= q < seg_pref[nseg]) of the concatenated stream: its point
// index, and the offset (dx, dy, dz) of its tile from the output tile.
__device__ __forceinline__ int p2g_candidate(const int *seg_start, const int *seg_pref, int nseg, int KT, int q,
                                             int &dx, int &dy, int &dz)
{
    int lo = 0, hi = nseg;  // seg_pref[lo] <= q < seg_pref[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (seg_pref[mid] <= q)
            lo = mid;
        else
            hi = mid;
    }
    const int side = KT + 1;
    dx = lo % side - KT;
    dy = (lo / side) % side - KT;
    dz = lo / (side * side) - KT;
    return seg_start[lo] + (q - seg_pref[lo]);
}

// The P bins of one (point, axis) from the first ceil(P/2) bins' polynomials:
// the window is even, so bin P-1-l at z is bin l at -z (w_{P-1-l}(z) =
// w_l(-z), and the Chebyshev fit inherits it), and both follow from the even
// and odd parts of bin l's polynomial, E(z^2) +- z O(z^2): half the Horner
// work of evaluating all P bins.  Packed FP32x2 over pairs of bins l.
template <int PC, int PS>
__device__ __forceinline__ void window_bins_sym(const float *coef, int nd, float zz, float (&pv)[PS])
{
    constexpr int NH = (PC + 1) / 2, NQ = (NH + 1) / 2;  // bins evaluated; their float2 pairs
    const float zsq = zz * zz;
    const float2 s2 = make_float2(zsq, zsq), z2 = make_float2(zz, zz), nz2 = make_float2(-zz, -zz);
    const int je = (nd - 1) & ~1, jo = ((nd - 1) & 1) ? nd - 1 : nd - 2;  // top even and odd powers
    float2 ev[NQ], od[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        ev[q] = *(const float2 *)(coef + je * PS + 2 * q);
        od[q] = jo >= 1 ? *(const float2 *)(coef + jo * PS + 2 * q) : make_float2(0.f, 0.f);
    }
    for (int j = je - 2; j >= 0; j -= 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            ev[q] = __ffma2_rn(ev[q], s2, *(const float2 *)(coef + j * PS + 2 * q));
    }
    for (int j = jo - 2; j >= 1; j -= 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            od[q] = __ffma2_rn(od[q], s2, *(const float2 *)(coef + j * PS + 2 * q));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float2 lo = __ffma2_rn(z2, od[q], ev[q]), hi = __ffma2_rn(nz2, od[q], ev[q]);
        const int l0 = 2 * q, l1 = 2 * q + 1;
        if (l0 < NH) {
            pv[l0] = lo.x;
            pv[PC - 1 - l0] = l0 < PC - 1 - l0 ? hi.x : pv[l0];
        }
        if (l1 < NH) {
            pv[l1] = lo.y;
            pv[PC - 1 - l1] = l1 < PC - 1 - l1 ? hi.y : pv[l1];
        }
    }
}

}  // namespace ewg
