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

}  // namespace ewg
