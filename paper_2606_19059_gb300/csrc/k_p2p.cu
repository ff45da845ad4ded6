// k_p2p.cu -- step a1: the near-field (P2P) sum of Sec. 2.1,
//
//   u^N_i = sum_j sum_p G^N(x_i - x_j + p) f_j   over 0 < |r| <= rc
//           - (4 xi / sqrt(pi)) sum_{j : r = 0} f_j,
//
// the last term removing the far part of every pair skipped at r = 0 (the
// self term for j = i; coincident points otherwise, Sec. 2).  The Hasimoto
// kernel of eq. (g-near) is written as
//   G^N f = (A - B) f + (A + B) r (r.f) / r^2,
//   A = erfc(xi r) / r,   B = (2 xi / sqrt(pi)) e^{-xi^2 r^2}.
//
// Work decomposition (prior art: the shared-memory 1-D variant of Sec. 3.1):
// one warp per chunk of <= 32 targets of one cell, one lane per target, and
// warps of a block fully independent (no block barrier: a warp waiting on its
// neighbours' pair counts would idle).  The sources of the colleague cells
// (for K = 1: those of their half-cell sub-cells that come within rc of the
// warp's target bounding box, about half the colleague volume) are
// concatenated into one stream that goes through the warp's own shared-memory
// tiles (FP32: a ring of two 64-source tiles; FP64: one tile of 128).  Per
// tile a lane first tests every candidate and records the in-range ones in a
// bit mask (phase 1, uniform across the warp; FP32 tests in FP16x2 with a
// safety margin), then walks its own set bits (phase 2).  Only in-range pairs
// are evaluated: about one candidate in five is in range, so a warp evaluating
// every candidate for all lanes would idle most lanes in the expensive branch.
//
// FP32 coordinates are cell-local in cell units and split hi + lo, hi on a
// 2^-20 lattice: colleague offsets are integers, so hi differences are exact
// and r = (hi_t - hi_s) + (lo_t - lo_s) keeps close pairs accurate to a few
// ulp of |r| (a plain FP32 coordinate would carry eps * cell).  FP64 uses
// cell-local coordinates in length units.
//
// erfc: FP64 uses the paper's rational erf(x)/x (Sec. 4) with erfc(x)/x =
// 1/x - erf(x)/x.  FP32 uses erfcx(x) = e^{x^2} erfc(x) as a polynomial in
// t = 1/(1 + x/2) times the e^{-x^2} the Gaussian term needs anyway (see
// fit_erf.py); the tight-tolerance form keeps the paper's form with a
// polynomial erf(x)/x below x = 1, where 1/r dominates.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "erf_rational.h"
#include "internal.h"

namespace ewg {
namespace {

__constant__ float c_erfcx32[ERFCX_F32_N];
__constant__ float c_erfxs32[ERFX_SMALL_N];
__constant__ double c_erfp64[ERF_RAT_F64_N];
__constant__ double c_erfq64[ERF_RAT_F64_N];

constexpr int kTile = 128;  // sources per staged tile = bits of the two masks

struct P2PArgs {
    const void *npos, *nfrc;  // FP64: cell-local positions, forces (4-vectors)
    const void *nrec;         // FP32: 32-byte records (lo.xyz, f.xyz, hi lattice)
    const void *nflo;         // double-single: the forces' FP32 rounding errors (float4)
    const int32_t *startn, *item_off, *permn;
    void *un;
    int nc, K, ncells;
    double cell, rc, xi;
};

__device__ __forceinline__ float fast_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fast_ex2(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct F32Const {
    float rc2, rc2_half, rcm, xi, nxi2log2e, nxi2log2e_lo, c2, selfc;
    // pairs with r^2 <= r1sq are left out (the double-single pass of a split
    // near field takes them); -1 when nothing is left out
    float r1sq;
};

// Squared pair distance (cell units) exactly as every FP32 pair form and the
// split near field's classification compute it, so that the FP32 and the
// double-single pass see the same r^2 for the same pair.
__device__ __forceinline__ float pair_r2(float dx, float dy, float dz)
{
    return fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz)));
}

__constant__ float c_exp2f32[EXP2_F32_N];

// e^{-xi^2 r^2} = 2^y, y = (r2 + r2lo) * (chi + clo) kept as y_hi + y_lo (the
// product's rounding recovered by an FMA), reduced to 2^f, |f| <= 1/2, by a minimax
// polynomial (fit_erf.py) and scaled by 2^n through the exponent bits.  About
// one ulp, where the hardware approximation and the FP32 rounding of y would
// each cost a few.  Valid for -125 <= y <= 0 (here y >= -50).
__device__ __forceinline__ float exp2_accurate(float r2, float r2lo, float chi, float clo)
{
    const float yh = r2 * chi;
    const float yl = fmaf(r2, chi, -yh) + fmaf(r2lo, chi, r2 * clo);
    const float n = rintf(yh);
    const float f = (yh - n) + yl;
    float p = c_exp2f32[EXP2_F32_N - 1];
#pragma unroll
    for (int q = EXP2_F32_N - 2; q >= 0; --q)
        p = fmaf(p, f, c_exp2f32[q]);
    return __int_as_float(__float_as_int(p) + ((int)n << 23));
}

// Kahan-compensated FP32 accumulation: s + c carries the sum to about one
// rounding of the largest partial, whatever the number of terms.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// One FP32 in-range candidate (cell units) at d = x_target - x_source, force
// f.  KAHAN selects the tight-tolerance form (tol < 1e-6): compensated
// accumulation (a blob point sums thousands of terms, and plain FP32 sums lose
// ~eps sqrt(n/2)), Newton-refined reciprocals and the accurate exponential
// above.
template <bool KAHAN, typename Acc>
__device__ __forceinline__ void pair_f32(float dx, float dy, float dz, const float3 &f,
                                         const F32Const &k, Acc &ax, Acc &ay, Acc &az)
{
    float r2 = pair_r2(dx, dy, dz);
    if (r2 > k.rc2 || r2 <= k.r1sq)
        return;
    if (r2 == 0.0f) {  // self or coincident point: the pair's far part comes out
        if constexpr (KAHAN) {
            ax.add(-k.selfc * f.x);
            ay.add(-k.selfc * f.y);
            az.add(-k.selfc * f.z);
        } else {
            ax = fmaf(-k.selfc, f.x, ax);
            ay = fmaf(-k.selfc, f.y, ay);
            az = fmaf(-k.selfc, f.z, az);
        }
        return;
    }
    // tight form: the rounding error of r2 as well, r2 + r2lo exact to ~2^-48
    // relative -- e^{-x^2} multiplies the relative error of r2 by x^2 (up to
    // ~25 at the cutoff), which would otherwise dominate the term's error
    float r2lo = 0.0f;
    if constexpr (KAHAN) {
        // _rn intrinsics: no contraction into FMAs, so each two-sum is exact
        const float px = __fmul_rn(dx, dx), py = __fmul_rn(dy, dy), pz = __fmul_rn(dz, dz);
        const float ex = fmaf(dx, dx, -px), ey = fmaf(dy, dy, -py), ez = fmaf(dz, dz, -pz);
        const float s1 = __fadd_rn(px, py), b1 = __fsub_rn(s1, px);
        const float e1 = __fadd_rn(__fsub_rn(px, __fsub_rn(s1, b1)), __fsub_rn(py, b1));
        const float s2 = __fadd_rn(s1, pz), b2 = __fsub_rn(s2, s1);
        const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, b2)), __fsub_rn(pz, b2));
        r2lo = ((ex + ey) + (ez + e1)) + e2 + __fsub_rn(s2, r2);
    }
    float rinv = rsqrtf(r2);
    if constexpr (KAHAN) {  // one Newton step: rinv *= 1 + (1 - r2 rinv^2) / 2
        float e = fmaf(-r2 * rinv, rinv, 1.0f);
        rinv = fmaf(0.5f * rinv, e, rinv);
    }
    float x = k.xi * (r2 * rinv);
    float E;  // e^{-xi^2 r^2}
    if constexpr (KAHAN)
        E = exp2_accurate(r2, r2lo, k.nxi2log2e, k.nxi2log2e_lo);
    else
        E = fast_ex2(r2 * k.nxi2log2e);
    float A;                               // erfc(xi r) / r
    // the tight form keeps 1/r exact for close pairs (small-x branch); the
    // bulk form takes erfcx on all of [0, 6], ~3e-7 relative in FP32
    if (KAHAN && x < (float)ERFX_SMALL_X32) {
        float t = x * x;
        float p = c_erfxs32[ERFX_SMALL_N - 1];
#pragma unroll
        for (int q = ERFX_SMALL_N - 2; q >= 0; --q)
            p = fmaf(p, t, c_erfxs32[q]);
        A = fmaf(-k.xi, p, rinv);          // 1/r - xi erf(x)/x
    } else {
        float d = fmaf((float)ERFCX_C32, x, 1.0f);
        float tt = fast_rcp(d);
        if constexpr (KAHAN)
            tt = fmaf(tt, fmaf(-d, tt, 1.0f), tt);
        float p = c_erfcx32[ERFCX_F32_N - 1];
#pragma unroll
        for (int q = ERFCX_F32_N - 2; q >= 0; --q)
            p = fmaf(p, tt, c_erfcx32[q]);
        A = (E * (tt * p)) * rinv;         // e^{-x^2} erfcx(x) / r
    }
    float B = k.c2 * E;
    float amb = A - B, apb = A + B;
    float rf = fmaf(dx, f.x, fmaf(dy, f.y, dz * f.z));
    float co = apb * rf * (rinv * rinv);
    if constexpr (KAHAN) {
        ax.add(fmaf(amb, f.x, co * dx));
        ay.add(fmaf(amb, f.y, co * dy));
        az.add(fmaf(amb, f.z, co * dz));
    } else {
        ax = fmaf(amb, f.x, fmaf(co, dx, ax));
        ay = fmaf(amb, f.y, fmaf(co, dy, ay));
        az = fmaf(amb, f.z, fmaf(co, dz, az));
    }
}

__device__ __forceinline__ float fast_rsqrt(float x)  // x >= 1e-30: no denormal inputs
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Bulk form without branches, two pairs at once (every source the bit walk
// yields runs the same instructions): the pairs' scalar factors go through
// packed FP32x2 arithmetic, one instruction for both pairs.  Returns the two
// terms.  In range (0 < r2 <= rc2): the kernel term.  r2 = 0: the far part of
// the skipped pair, -selfc f (r2 + 1e-30 keeps 1/r finite there, and d = 0
// zeroes the r (r.f) part).  Beyond rc (what passes the FP16 test's margin,
// and the dummy entries): r2 is replaced by 1e30, for which e^{-xi^2 r^2}, and
// with it every factor of the term, is exactly 0.  SPLIT (the outer pass of a
// split near field): pairs with r2 <= r1sq, r = 0 among them, are left to the
// double-single pass and get r2 = 1e30 too.
template <bool SPLIT>
__device__ __forceinline__ void pair2_f32_bulk(const float3 &d0, const float3 &f0, const float3 &d1,
                                               const float3 &f1, const F32Const &k, float3 &c0,
                                               float3 &c1)
{
    const float ra = pair_r2(d0.x, d0.y, d0.z);
    const float rb = pair_r2(d1.x, d1.y, d1.z);
    const bool ina = ra <= k.rc2 && (!SPLIT || ra > k.r1sq), inb = rb <= k.rc2 && (!SPLIT || rb > k.r1sq);
    const float2 r2s = make_float2(ina ? ra + 1e-30f : 1e30f, inb ? rb + 1e-30f : 1e30f);
    const float2 rinv = make_float2(fast_rsqrt(r2s.x), fast_rsqrt(r2s.y));
    const float2 x = __fmul2_rn(make_float2(k.xi, k.xi), __fmul2_rn(r2s, rinv));
    const float2 ea = __fmul2_rn(r2s, make_float2(k.nxi2log2e, k.nxi2log2e));
    const float2 E = make_float2(fast_ex2(ea.x), fast_ex2(ea.y));
    const float2 den = __ffma2_rn(make_float2((float)ERFCX_C32, (float)ERFCX_C32), x, make_float2(1.f, 1.f));
    const float2 tt = make_float2(fast_rcp(den.x), fast_rcp(den.y));
    float2 p = make_float2(c_erfcx32[ERFCX_F32_N - 1], c_erfcx32[ERFCX_F32_N - 1]);
#pragma unroll
    for (int q = ERFCX_F32_N - 2; q >= 0; --q)
        p = __ffma2_rn(p, tt, make_float2(c_erfcx32[q], c_erfcx32[q]));
    const float2 Ar = __fmul2_rn(__fmul2_rn(tt, p), rinv);  // erfcx(x) / r: A = E Ar
    const float2 B = __fmul2_rn(make_float2(k.c2, k.c2), E);
    const float2 nB = __fmul2_rn(make_float2(-k.c2, -k.c2), E);
    float2 amb = __ffma2_rn(E, Ar, nB);
    const float2 apb = __ffma2_rn(E, Ar, B);
    if constexpr (!SPLIT) {
        amb.x = ra == 0.0f ? -k.selfc : amb.x;
        amb.y = rb == 0.0f ? -k.selfc : amb.y;
    }
    const float2 rf = make_float2(fmaf(d0.x, f0.x, fmaf(d0.y, f0.y, d0.z * f0.z)),
                                  fmaf(d1.x, f1.x, fmaf(d1.y, f1.y, d1.z * f1.z)));
    const float2 co = __fmul2_rn(__fmul2_rn(apb, rf), __fmul2_rn(rinv, rinv));
    c0 = make_float3(fmaf(amb.x, f0.x, co.x * d0.x), fmaf(amb.x, f0.y, co.x * d0.y),
                     fmaf(amb.x, f0.z, co.x * d0.z));
    c1 = make_float3(fmaf(amb.y, f1.x, co.y * d1.x), fmaf(amb.y, f1.y, co.y * d1.y),
                     fmaf(amb.y, f1.z, co.y * d1.z));
}

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

constexpr int kWarps = 4;       // independent warps per block
constexpr int kMaxSeg = 288;    // K = 1: the 8 x 6 x 6 sub-cells around a group; K = 2: 125 cells

// Per-warp shared state: the colleague source ranges kept for this warp,
// concatenated into one stream (prefix offsets), and one staged tile of it.
template <typename Tile>
struct WarpSmem {
    Tile tile;
    int seg_start[kMaxSeg];
    int seg_pref[kMaxSeg + 1];
    uint16_t seg_off[kMaxSeg];  // colleague cell offset, (dx+2) | (dy+2) << 4 | (dz+2) << 8
};

// Work item = (cell group, chunk of <= 32 targets) handled by one warp: c is
// the group's first cell, targets [tb, te); those from tsplit on lie in the
// group's second cell (one cell further in x).
__device__ __forceinline__ bool find_item(const P2PArgs &a, int item, int &c, int &tb, int &te, int &tsplit)
{
    const int ng = p2p_groups(a.nc, a.K);
    if (item >= a.item_off[ng])
        return false;
    int lo = 0, hi = ng;  // item_off[lo] <= item < item_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a.item_off[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    int ncg;
    c = p2p_group_cell(lo, a.nc, a.K, ncg);
    const int chunk = item - a.item_off[lo];
    const int nch = a.item_off[lo + 1] - a.item_off[lo];
    const int t0 = a.startn[c * kSub3], t1 = a.startn[(c + ncg) * kSub3];
    tsplit = ncg > 1 ? a.startn[(c + 1) * kSub3] : t1;
    const int per = (t1 - t0 + nch - 1) / nch;
    tb = t0 + chunk * per;
    te = min(t1, tb + per);
    return true;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Build the warp's source stream for the group starting at cell c.  K = 1: the
// 8 x 6 x 6 sub-cells (half a cell wide) of the colleague cells of the group's
// two cells, keeping those whose box comes within rc of the bounding box
// [blo, bhi] of the warp's targets -- the warp's 32 targets sit in a few
// sub-cells, so most of the colleague volume is out of reach.  K = 2 (small
// boxes): the 125 colleague cells, all kept.  Coordinates are local to cell c;
// `hw` is half a cell in their units and `rcm` the cutoff plus a margin.
// Empty segments are dropped.
template <typename WS>
__device__ __forceinline__ int build_segments(const P2PArgs &a, int c, WS &ws, int lane, float3 blo,
                                              float3 bhi, float hw, float rcm)
{
    const int K = a.K, nc = a.nc;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const bool sub = K == 1;
    const int side = 2 * K + 1;
    const int nent = sub ? 288 : side * side * side;
    int carry = 0, kept = 0;
    for (int s0 = 0; s0 < nent; s0 += 32) {
        const int s = s0 + lane;
        bool keep = false;
        int start = 0, len = 0, off = 0;
        if (s < nent) {
            int dx, dy, dz, key_lo, key_hi;
            if (sub) {
                // half-cell index relative to cell c's corner: -2..5 in x,
                // -2..3 in y and z
                const int ix = s % 8 - 2, iy = (s / 8) % 6 - 2, iz = s / 48 - 2;
                const float gx = fmaxf(0.f, fmaxf(ix * hw - bhi.x, blo.x - (ix + 1) * hw));
                const float gy = fmaxf(0.f, fmaxf(iy * hw - bhi.y, blo.y - (iy + 1) * hw));
                const float gz = fmaxf(0.f, fmaxf(iz * hw - bhi.z, blo.z - (iz + 1) * hw));
                keep = gx * gx + gy * gy + gz * gz <= rcm * rcm;
                dx = ix >> 1;  // floor division by 2
                dy = iy >> 1;
                dz = iz >> 1;
                const int sc = ((iz & 1) * kSub + (iy & 1)) * kSub + (ix & 1);
                const int nb = (wrap(cz + dz, nc) * nc + wrap(cy + dy, nc)) * nc + wrap(cx + dx, nc);
                key_lo = nb * kSub3 + sc;
                key_hi = key_lo + 1;
            } else {
                dx = s % side - K;
                dy = (s / side) % side - K;
                dz = s / (side * side) - K;
                keep = true;
                const int nb = (wrap(cz + dz, nc) * nc + wrap(cy + dy, nc)) * nc + wrap(cx + dx, nc);
                key_lo = nb * kSub3;
                key_hi = key_lo + kSub3;
            }
            if (keep) {
                start = a.startn[key_lo];
                len = a.startn[key_hi] - start;
                keep = len > 0;
                off = (dx + 2) | ((dy + 2) << 4) | ((dz + 2) << 8);
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        int v = keep ? len : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o)
                v += u;
        }
        if (keep) {
            const int pos = kept + __popc(ball & ((1u << lane) - 1u));
            ws.seg_start[pos] = start;
            ws.seg_off[pos] = (uint16_t)off;
            ws.seg_pref[pos + 1] = carry + v;
        }
        carry += __shfl_sync(0xffffffffu, v, 31);
        kept += __popc(ball);
    }
    if (lane == 0)
        ws.seg_pref[0] = 0;
    __syncwarp();
    return kept;
}

// Segment of stream element q (binary search over the prefix offsets).
template <typename WS>
__device__ __forceinline__ int seg_of(const WS &ws, int nseg, int q)
{
    int lo = 0, hi = nseg;  // seg_pref[lo] <= q < seg_pref[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (ws.seg_pref[mid] <= q)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Stream element q of segment sg: its index in the sorted arrays and the
// colleague cell offset.
template <typename WS>
__device__ __forceinline__ int seg_element(const WS &ws, int sg, int q, int &dx, int &dy, int &dz)
{
    const int off = ws.seg_off[sg];
    dx = (off & 15) - 2;
    dy = ((off >> 4) & 15) - 2;
    dz = ((off >> 8) & 15) - 2;
    return ws.seg_start[sg] + (q - ws.seg_pref[sg]);
}

// Source q of the stream: its index in the sorted arrays and colleague offset.
template <typename WS>
__device__ __forceinline__ int locate(const WS &ws, int nseg, int q, int &dx, int &dy, int &dz)
{
    return seg_element(ws, seg_of(ws, nseg, q), q, dx, dy, dz);
}

constexpr float kFarHalf = 64.0f;  // FP16 dummy source: r^2 ~ 1e4, finite and never within rc

// FP16 phase-1 threshold on r^2 (cell units, cutoff rcc <= 2 cells).  In FP16
// a source coordinate (|v| < 4) is off by <= 2^-10, a target's (in [0, 2): a
// cell group's second cell) by <= 2^-11, their difference adds <= 2^-11: |d|
// by <= 2e-3 per component, r^2 by <= 7e-3 rcc; the FP16 sums add <= 3e-3 and
// rounding the threshold <= 2e-3.  0.008 (rcc + rcc^2) + 0.002 covers that
// about twice over, so no pair within rc fails the test; the few beyond it
// that pass are dropped later.
__host__ __device__ inline float half_threshold(double rcc)
{
    return (float)(rcc * rcc + 0.008 * (rcc + rcc * rcc) + 0.002);
}

// FP32 kernel: tiles of 64 sources, two staged at once (a ring of two slots),
// so a lane may run up to one tile ahead of the slowest lane of its warp: the
// warp's pair iterations then follow the busiest lane's total over the whole
// stream instead of the sum over tiles of each tile's busiest lane (about a
// fifth fewer for Poisson-like in-range counts of ~11 per lane and tile).
constexpr int kT32 = 64;

// FP16x2 phase 1 over one 64-source tile: each shared load brings sources k
// and k + 32, one FP16x2 distance test covers both, and one AND-OR files the
// two results.  Word w (0, 1) gets bit b < 16 for source 16 w + b and bit
// 16 + b for source 32 + 16 w + b.  Coordinates are cell-local with |value| <= 3,
// so FP16 keeps their differences to ~2^-10.
__device__ __forceinline__ void phase1_words(const uint4 *sh, __half2 tx, __half2 ty, __half2 tz,
                                             __half2 lim, unsigned &w0, unsigned &w1)
{
    unsigned acc[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < kT32 / 2; ++k) {
        const uint4 v = sh[k];
        const __half2 dx = __hsub2(tx, *(const __half2 *)&v.x);
        const __half2 dy = __hsub2(ty, *(const __half2 *)&v.y);
        const __half2 dz = __hsub2(tz, *(const __half2 *)&v.z);
        const __half2 r2 = __hfma2(dx, dx, __hfma2(dy, dy, __hmul2(dz, dz)));
        acc[k >> 4] |= __hle2_mask(r2, lim) & ((1u << (k & 15)) | (1u << (16 + (k & 15))));
    }
    w0 = acc[0];
    w1 = acc[1];
}

// Highest set bit of w (-1 for w = 0), and w with bit b cleared (w itself for
// b = -1: PTX clamps the shift count, so 1 << b is then 0).
__device__ __forceinline__ int bfind(unsigned w)
{
    int b;
    asm("bfind.u32 %0, %1;" : "=r"(b) : "r"(w));
    return b;
}
__device__ __forceinline__ unsigned clear_bit(unsigned w, int b)
{
    unsigned m;
    asm("shl.b32 %0, %1, %2;" : "=r"(m) : "r"(1u), "r"(b));
    return w ^ m;
}

// FP32 ring layout: the two staged tiles are four groups of 33 entries, group
// g = 2 slot + w for word w of the slot's masks: entry 33 g is a dummy source
// (far away, zero force: its term is exactly 0), entries 33 g + 1 + b the
// sources of bit b.
constexpr int kGrp = 33;

// A lane's in-range bits of the staged tiles as a queue of 32-bit words in pop
// order; w0 is being popped and g is its group.  pop() shifts the queue by a
// word when w0 is used up (a zero enters at the back), then takes w0's highest
// bit -- or the group's dummy when w0 is empty -- so a pop costs a few selects
// and one bit search whatever the mask.
struct BitQueue {
    unsigned w0, w1, w2, w3;
    int g;
    __device__ __forceinline__ void shift_if(bool e)
    {
        w0 = e ? w1 : w0;
        w1 = e ? w2 : w1;
        w2 = e ? w3 : w2;
        w3 = e ? 0u : w3;
        g = e ? ((g + 1) & 3) : g;
    }
    __device__ __forceinline__ int pop()
    {
        shift_if(w0 == 0u);
        const int b = bfind(w0);
        w0 = clear_bit(w0, b);
        return kGrp * g + 1 + b;
    }
    // in-range sources of the cursor's tile still queued (the cursor is on the
    // tile's first word when g is even)
    __device__ __forceinline__ int pending() const
    {
        return __popc(w0) + ((g & 1) ? 0 : __popc(w1));
    }
};

// Next set bit of the 128-bit mask (m0 first), without divergent branches.
__device__ __forceinline__ int next_bit(unsigned long long &m0, unsigned long long &m1)
{
    const bool first = m0 != 0ull;
    unsigned long long m = first ? m0 : m1;
    const int k = __ffsll((long long)m) - 1 + (first ? 0 : 64);
    m &= m - 1;
    m0 = first ? m : m0;
    m1 = first ? m1 : m;
    return k;
}

// FP32 ring entries (groups as above): sa = (hi + colleague offset, lo.x),
// sb = (lo.y, lo.z, f.x, f.y), sc = f.z -- 36 bytes a source, read by phase 2 --
// and per slot the FP16 copy of the positions read by phase 1.
struct TileF32 {
    float4 sa[4 * kGrp];
    float4 sb[4 * kGrp];
    float sc[4 * kGrp];
    uint4 sh[2][kT32 / 2];
};

// FP64 tile of 128 sources: positions (hi + colleague offset, length units)
// and forces as packed double triples, and the FP16 copy of the positions in
// cell units for phase 1 (sources k and k + 64 per entry).
struct TileF64 {
    double3 sp[kTile];
    double3 sf[kTile];
    uint4 sh[kTile / 2];
};
// FP16x2 phase 1 over one 128-source tile (FP64 kernel): entry k holds
// sources k and k + 64; word w of the result holds entries 16 w .. 16 w + 15,
// bit b < 16 source 16 w + b, bit 16 + b source 64 + 16 w + b (half_slot_128
// inverts this).  Same coordinates (cell units, |value| <= 3) and threshold as
// the FP32 kernel.
__device__ __forceinline__ void phase1_half_128(const uint4 *sh, __half2 tx, __half2 ty, __half2 tz,
                                                __half2 lim, unsigned long long &m0,
                                                unsigned long long &m1)
{
    unsigned acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < kTile / 2; ++k) {
        const uint4 v = sh[k];
        const __half2 dx = __hsub2(tx, *(const __half2 *)&v.x);
        const __half2 dy = __hsub2(ty, *(const __half2 *)&v.y);
        const __half2 dz = __hsub2(tz, *(const __half2 *)&v.z);
        const __half2 r2 = __hfma2(dx, dx, __hfma2(dy, dy, __hmul2(dz, dz)));
        acc[k >> 4] |= __hle2_mask(r2, lim) & ((1u << (k & 15)) | (1u << (16 + (k & 15))));
    }
    m0 = ((unsigned long long)acc[1] << 32) | acc[0];
    m1 = ((unsigned long long)acc[3] << 32) | acc[2];
}

__device__ __forceinline__ int half_slot_128(int p)
{
    return ((p >> 5) << 4) + (p & 15) + ((p & 16) << 2);
}

// FP64 pair without branches (two in flight per lane): in range (0 < r2 <=
// rc2) the kernel term, r2 = 0 the removed far part, else nothing.  The
// paper's erf(x)/x rational; erfc(x) is taken as 0 past x = 7 (4e-23).
__device__ __forceinline__ double3 pair_f64_bulk(double dx, double dy, double dz, const double3 &f,
                                                 double rc2, double xi, double xi2, double c2,
                                                 double selfc)
{
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const bool in = r2 <= rc2 && r2 > 0.0;
    const double r2s = in ? r2 : 1.0;
    const double rinv = rsqrt(r2s);
    const double x = xi * (r2s * rinv);
    const double z = fma(fmin(x, ERF_RAT_X64), 2.0 / ERF_RAT_X64, -1.0);
    double P = c_erfp64[ERF_RAT_F64_N - 1], Q = c_erfq64[ERF_RAT_F64_N - 1];
#pragma unroll
    for (int q = ERF_RAT_F64_N - 2; q >= 0; --q) {
        P = fma(P, z, c_erfp64[q]);
        Q = fma(Q, z, c_erfq64[q]);
    }
    const double A = x < ERF_RAT_X64 ? rinv - xi * (P / Q) : 0.0;  // erfc(x)/r
    const double B = c2 * exp(-xi2 * r2s);
    const double amb = A - B, apb = A + B;
    const double rf = fma(dx, f.x, fma(dy, f.y, dz * f.z));
    const double co = apb * rf * (rinv * rinv);
    const double sc = r2 == 0.0 ? -selfc : 0.0;
    return make_double3(in ? fma(amb, f.x, co * dx) : sc * f.x, in ? fma(amb, f.y, co * dy) : sc * f.y,
                        in ? fma(amb, f.z, co * dz) : sc * f.z);
}

using WsF32 = WarpSmem<TileF32>;
using WsF64 = WarpSmem<TileF64>;

// FP32 record -> hi (21-bit lattice integers times 2^-20), lo and force.
__device__ __forceinline__ void unpack_rec(const float4 &A, const float4 &B, float3 &hi, float3 &lo,
                                           float3 &f)
{
    const unsigned w0 = __float_as_uint(B.z), w1 = __float_as_uint(B.w);
    const unsigned qx = w0 & 0x1FFFFFu, qy = (w0 >> 21) | ((w1 & 0x3FFu) << 11), qz = w1 >> 10;
    hi = make_float3((float)(int)qx * (1.f / 1048576.f), (float)(int)qy * (1.f / 1048576.f),
                     (float)(int)qz * (1.f / 1048576.f));
    lo = make_float3(A.x, A.y, A.z);
    f = make_float3(A.w, B.x, B.y);
}

// Stage tile `tile` of the warp's stream (strided: elements tile, tile +
// ntile, ...) into ring slot `slot`; each lane stages sources lane and
// lane + 32, at the entries of their phase-1 bits, and packs their FP16 copy.
// Tiles are staged in order, so a lane's element q is its previous one plus 1:
// sg[h] follows its segment with at most one step (segments are never empty),
// the binary search only for tile 0.
__device__ __forceinline__ void stage_f32(const P2PArgs &a, WsF32 &ws, int nseg, int slot,
                                          int tile, int ntile, int total, int lane, int (&sg)[2])
{
    const float4 *rec = (const float4 *)a.nrec;
    float3 hp[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h, q = tile + k * ntile;
        if (q < total) {
            if (tile == 0)
                sg[h] = seg_of(ws, nseg, q);
            else if (ws.seg_pref[sg[h] + 1] <= q)
                ++sg[h];
            int dx, dy, dz;
            const int j = seg_element(ws, sg[h], q, dx, dy, dz);
            const float4 A = rec[2 * j], B = rec[2 * j + 1];
            float3 hi, lo, f;
            unpack_rec(A, B, hi, lo, f);
            // exact: integer colleague offsets, hi on a 2^-20 lattice
            hp[h] = make_float3(hi.x + (float)dx, hi.y + (float)dy, hi.z + (float)dz);
            const int e = kGrp * (2 * slot + (lane >> 4)) + 1 + (lane & 15) + 16 * h;
            ws.tile.sa[e] = make_float4(hp[h].x, hp[h].y, hp[h].z, lo.x);
            ws.tile.sb[e] = make_float4(lo.y, lo.z, f.x, f.y);
            ws.tile.sc[e] = f.z;
        } else {
            hp[h] = make_float3(kFarHalf, kFarHalf, kFarHalf);
        }
    }
    const __half2 hx = __floats2half2_rn(hp[0].x, hp[1].x);
    const __half2 hy = __floats2half2_rn(hp[0].y, hp[1].y);
    const __half2 hz = __floats2half2_rn(hp[0].z, hp[1].z);
    ws.tile.sh[slot][lane] = make_uint4(*(const unsigned *)&hx, *(const unsigned *)&hy,
                                        *(const unsigned *)&hz, 0u);
}

// One work item (a chunk of <= 32 targets of one cell) by one warp.  Rounds
// over the tiles: round o runs until every lane has evaluated its in-range
// sources of tile o -- the busiest lane's count, known up front -- while lanes
// done early go on into tile o + 1; then tile o + 2 takes tile o's slot.
// KAHAN: compensated partial sums, flushed into FP64 totals every round, of
// the tight pair form -- or, with BULK2 (the outer pass of a split near
// field), of the two-pair bulk form without the pairs within r1.
template <bool KAHAN, bool BULK2 = false>
__device__ __forceinline__ bool p2p_f32_run(const P2PArgs &a, const F32Const &kc, int item, WsF32 &ws, int lane,
                                            int &t_out, bool &act_out,
                                            typename std::conditional<KAHAN, double, float>::type (&u)[3])
{
    using Tot = typename std::conditional<KAHAN, double, float>::type;
    int c, tb, te, tsplit;
    if (!find_item(a, item, c, tb, te, tsplit))
        return false;  // whole warp: no block-wide barrier follows
    const int t = tb + lane;
    const bool active = t < te;
    t_out = t;
    act_out = active;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
    if (active) {
        const float4 *rec = (const float4 *)a.nrec;
        float3 hi, lo, f;
        unpack_rec(rec[2 * t], rec[2 * t + 1], hi, lo, f);
        // relative to cell c: the group's second cell is one cell on in x (exact)
        th = make_float4(hi.x + (t >= tsplit ? 1.f : 0.f), hi.y, hi.z, 0.f);
        tl = make_float4(lo.x, lo.y, lo.z, 0.f);
    }
    // the warp's target bounding box (hi parts; the margin covers lo)
    const float3 blo = make_float3(warp_min(active ? th.x : 1e30f), warp_min(active ? th.y : 1e30f),
                                   warp_min(active ? th.z : 1e30f));
    const float3 bhi = make_float3(warp_max(active ? th.x : -1e30f),
                                   warp_max(active ? th.y : -1e30f),
                                   warp_max(active ? th.z : -1e30f));
    const int nseg = build_segments(a, c, ws, lane, blo, bhi, 0.5f, kc.rcm);
    const int total = ws.seg_pref[nseg];
    // tile t holds the stream elements t, t + ntiles, t + 2 ntiles, ...: each
    // tile samples the whole neighbourhood, so the lanes' in-range counts per
    // tile are even
    const int ntile = (total + kT32 - 1) / kT32;
    const __half2 tx = __float2half2_rn(th.x), ty = __float2half2_rn(th.y),
                  tz = __float2half2_rn(th.z), lim = __float2half2_rn(kc.rc2_half);
    if (lane < 4) {  // the groups' dummy sources
        ws.tile.sa[kGrp * lane] = make_float4(1e3f, 1e3f, 1e3f, 0.f);
        ws.tile.sb[kGrp * lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        ws.tile.sc[kGrp * lane] = 0.f;
    }
    int sg[2] = {0, 0};
    for (int tt = 0; tt < 2 && tt < ntile; ++tt)
        stage_f32(a, ws, nseg, tt, tt, ntile, total, lane, sg);
    __syncwarp();
    BitQueue q = {0u, 0u, 0u, 0u, 0};  // inactive lanes: empty throughout
    if (active) {
        if (ntile > 0)
            phase1_words(ws.tile.sh[0], tx, ty, tz, lim, q.w0, q.w1);
        if (ntile > 1)
            phase1_words(ws.tile.sh[1], tx, ty, tz, lim, q.w2, q.w3);
    }
    Tot ux = 0, uy = 0, uz = 0;
    for (int o = 0; o < ntile; ++o) {
        const int need = (int)__reduce_max_sync(0xffffffffu, (unsigned)q.pending());
        typename std::conditional<KAHAN, KSum, float>::type px{}, py{}, pz{};
        if constexpr (KAHAN && BULK2) {
            for (int it = 0; it < (need + 1) >> 1; ++it) {
                const int e0 = q.pop(), e1 = q.pop();
                const float4 s0 = ws.tile.sa[e0], b0 = ws.tile.sb[e0];
                const float4 s1 = ws.tile.sa[e1], b1 = ws.tile.sb[e1];
                const float f0 = ws.tile.sc[e0], f1 = ws.tile.sc[e1];
                float3 c0, c1;
                pair2_f32_bulk<true>(make_float3((th.x - s0.x) + (tl.x - s0.w), (th.y - s0.y) + (tl.y - b0.x),
                                                 (th.z - s0.z) + (tl.z - b0.y)),
                                     make_float3(b0.z, b0.w, f0),
                                     make_float3((th.x - s1.x) + (tl.x - s1.w), (th.y - s1.y) + (tl.y - b1.x),
                                                 (th.z - s1.z) + (tl.z - b1.y)),
                                     make_float3(b1.z, b1.w, f1), kc, c0, c1);
                px.add(c0.x);
                px.add(c1.x);
                py.add(c0.y);
                py.add(c1.y);
                pz.add(c0.z);
                pz.add(c1.z);
            }
        } else if constexpr (KAHAN) {
            for (int it = 0; it < need; ++it) {
                const int e = q.pop();
                const float4 s = ws.tile.sa[e], b = ws.tile.sb[e];
                // d = (hi diff, exact) + (lo diff)
                pair_f32<KAHAN>((th.x - s.x) + (tl.x - s.w), (th.y - s.y) + (tl.y - b.x),
                                (th.z - s.z) + (tl.z - b.y), make_float3(b.z, b.w, ws.tile.sc[e]),
                                kc, px, py, pz);
            }
        } else {
            // two pairs per iteration: independent chains for the scheduler
            for (int it = 0; it < (need + 1) >> 1; ++it) {
                const int e0 = q.pop(), e1 = q.pop();
                const float4 s0 = ws.tile.sa[e0], b0 = ws.tile.sb[e0];
                const float4 s1 = ws.tile.sa[e1], b1 = ws.tile.sb[e1];
                const float f0 = ws.tile.sc[e0], f1 = ws.tile.sc[e1];
                float3 c0, c1;
                pair2_f32_bulk<false>(make_float3((th.x - s0.x) + (tl.x - s0.w), (th.y - s0.y) + (tl.y - b0.x),
                                           (th.z - s0.z) + (tl.z - b0.y)),
                               make_float3(b0.z, b0.w, f0),
                               make_float3((th.x - s1.x) + (tl.x - s1.w), (th.y - s1.y) + (tl.y - b1.x),
                                           (th.z - s1.z) + (tl.z - b1.y)),
                               make_float3(b1.z, b1.w, f1), kc, c0, c1);
                // the two terms summed first: one rounding at the partial sum's
                // size per two pairs
                px += c0.x + c1.x;
                py += c0.y + c1.y;
                pz += c0.z + c1.z;
            }
        }
        if constexpr (KAHAN) {
            ux += (double)px.s + (double)px.c * -1.0;
            uy += (double)py.s + (double)py.c * -1.0;
            uz += (double)pz.s + (double)pz.c * -1.0;
        } else {
            ux += px;
            uy += py;
            uz += pz;
        }
        // every lane is past tile o: drop its used-up words, which leaves the
        // cursor in tile o + 1
        q.shift_if((q.g >> 1) == (o & 1));
        q.shift_if((q.g >> 1) == (o & 1));
        if (o + 2 < ntile) {  // slot o & 1 is free: tile o + 2 goes there
            __syncwarp();
            stage_f32(a, ws, nseg, o & 1, o + 2, ntile, total, lane, sg);
            __syncwarp();
            unsigned c0 = 0u, c1 = 0u;
            if (active)
                phase1_words(ws.tile.sh[o & 1], tx, ty, tz, lim, c0, c1);
            // queue its words behind tile o + 1's
            const bool odd = q.g & 1;
            q.w1 = odd ? c0 : q.w1;
            q.w2 = odd ? c1 : c0;
            q.w3 = odd ? 0u : c1;
        }
    }
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
    return true;
}

// One work item (a chunk of <= 32 targets) by one warp: the sums of
// p2p_f32_run, in length units, into the FP32 near result.
template <bool KAHAN>
__device__ __forceinline__ void p2p_f32_item(const P2PArgs &a, const F32Const &kc, float inv_cell,
                                             int item, WsF32 &ws, int lane)
{
    typename std::conditional<KAHAN, double, float>::type u[3];
    int t;
    bool active;
    if (!p2p_f32_run<KAHAN>(a, kc, item, ws, lane, t, active, u))
        return;
    if (active) {
        const int i = a.permn[t];
        float *un = (float *)a.un;
        un[3 * i] = (float)(u[0] * inv_cell);
        un[3 * i + 1] = (float)(u[1] * inv_cell);
        un[3 * i + 2] = (float)(u[2] * inv_cell);
    }
}


template <bool KAHAN>
__global__ void __launch_bounds__(kWarps * 32) k_p2p_f32(P2PArgs a, F32Const kc, float inv_cell)
{
    __shared__ WsF32 wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    p2p_f32_item<KAHAN>(a, kc, inv_cell, blockIdx.x * kWarps + warp, wsm[warp], lane);
}

__device__ __forceinline__ void p2p_f64_item(const P2PArgs &a, int item, WsF64 &ws, int lane)
{
    double3 *sp = ws.tile.sp, *sf = ws.tile.sf;
    uint4 *sh = ws.tile.sh;
    int c, tb, te, tsplit;
    if (!find_item(a, item, c, tb, te, tsplit))
        return;
    const dvec4 *npos = (const dvec4 *)a.npos, *nfrc = (const dvec4 *)a.nfrc;
    const int t = tb + lane;
    const bool active = t < te;
    dvec4 xt = {0.0, 0.0, 0.0, 0.0};
    if (active) {
        xt = npos[t];
        if (t >= tsplit)  // relative to cell c: the group's second cell
            xt.x += a.cell;
    }
    const double rc2 = a.rc * a.rc, xi = a.xi, xi2 = a.xi * a.xi;
    const double c2 = 2.0 * a.xi / sqrt(3.14159265358979323846), selfc = 2.0 * c2;
    const double inv_cell = 1.0 / a.cell, rcc = a.rc * inv_cell;
    const float3 blo = make_float3(warp_min(active ? (float)xt.x : 1e30f),
                                   warp_min(active ? (float)xt.y : 1e30f),
                                   warp_min(active ? (float)xt.z : 1e30f));
    const float3 bhi = make_float3(warp_max(active ? (float)xt.x : -1e30f),
                                   warp_max(active ? (float)xt.y : -1e30f),
                                   warp_max(active ? (float)xt.z : -1e30f));
    const int nseg = build_segments(a, c, ws, lane, blo, bhi, (float)(0.5 * a.cell),
                                    (float)(a.rc + 1e-3 * a.cell));
    const int total = ws.seg_pref[nseg];
    const int ntile = (total + kTile - 1) / kTile;  // strided tiles, as in k_p2p_f32
    // phase 1 in FP16 on cell-unit coordinates (the FP32 kernel's bound)
    const __half2 tx = __float2half2_rn((float)(xt.x * inv_cell)), ty = __float2half2_rn((float)(xt.y * inv_cell)),
                  tz = __float2half2_rn((float)(xt.z * inv_cell)),
                  lim = __float2half2_rn(half_threshold(rcc));
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int tile = 0; tile < ntile; ++tile) {
        const int n = (total - tile + ntile - 1) / ntile;
#pragma unroll
        for (int i = 0; i < kTile / 64; ++i) {
            float3 hp[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = lane + 32 * i + 64 * h, q = tile + k * ntile;
                if (k < n) {
                    int dx, dy, dz;
                    const int j = locate(ws, nseg, q, dx, dy, dz);
                    const dvec4 p = npos[j], f = nfrc[j];
                    const double3 pp = make_double3(p.x + dx * a.cell, p.y + dy * a.cell, p.z + dz * a.cell);
                    sp[k] = pp;
                    sf[k] = make_double3(f.x, f.y, f.z);
                    hp[h] = make_float3((float)(pp.x * inv_cell), (float)(pp.y * inv_cell),
                                        (float)(pp.z * inv_cell));
                } else {
                    hp[h] = make_float3(kFarHalf, kFarHalf, kFarHalf);
                }
            }
            const __half2 hx = __floats2half2_rn(hp[0].x, hp[1].x);
            const __half2 hy = __floats2half2_rn(hp[0].y, hp[1].y);
            const __half2 hz = __floats2half2_rn(hp[0].z, hp[1].z);
            sh[lane + 32 * i] = make_uint4(*(const unsigned *)&hx, *(const unsigned *)&hy,
                                           *(const unsigned *)&hz, 0u);
        }
        __syncwarp();
        unsigned long long m0 = 0ull, m1 = 0ull;
        if (active)
            phase1_half_128(sh, tx, ty, tz, lim, m0, m1);
        // two pairs per iteration: independent FP64 chains for the scheduler
        double px = 0.0, py = 0.0, pz = 0.0;
        while (__any_sync(0xffffffffu, (m0 | m1) != 0ull)) {
            double3 d[2], fv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                d[u] = make_double3(1e3, 0.0, 0.0);
                fv[u] = make_double3(0.0, 0.0, 0.0);
                if (m0 | m1) {
                    const int k = half_slot_128(next_bit(m0, m1));
                    const double3 s = sp[k];
                    d[u] = make_double3(xt.x - s.x, xt.y - s.y, xt.z - s.z);
                    fv[u] = sf[k];
                }
            }
            const double3 c0 = pair_f64_bulk(d[0].x, d[0].y, d[0].z, fv[0], rc2, xi, xi2, c2, selfc);
            const double3 c1 = pair_f64_bulk(d[1].x, d[1].y, d[1].z, fv[1], rc2, xi, xi2, c2, selfc);
            px += c0.x + c1.x;
            py += c0.y + c1.y;
            pz += c0.z + c1.z;
        }
        ux += px;
        uy += py;
        uz += pz;
        __syncwarp();
    }
    if (active) {
        const int i = a.permn[t];
        double *un = (double *)a.un;
        un[3 * i] = ux;
        un[3 * i + 1] = uy;
        un[3 * i + 2] = uz;
    }
}

__global__ void __launch_bounds__(kWarps * 32, 5) k_p2p_f64(P2PArgs a)
{
    __shared__ WsF64 wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    p2p_f64_item(a, blockIdx.x * kWarps + warp, wsm[warp], lane);
}

// ---- double-single near field ---------------------------------------------
// Values carried as unevaluated sums h + l of two FP32 numbers (|l| <= ulp(h)/2,
// ~44 significant bits): the FP32 pipe does ~64x the FP64 work per clock on
// this GPU, so FP32 pairs beat native FP64 for the tol 1e-8 near field.  The
// error-free transformations are the standard ones (Knuth's two-sum, Dekker's
// fast two-sum, the FMA two-product); the _rn intrinsics keep the compiler
// from contracting them into FMAs, which would break their exactness.
struct dsf {
    float h, l;
};

__device__ __forceinline__ dsf two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), v = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ dsf quick_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dsf ds_add(dsf x, dsf y)
{
    const dsf s = two_sum(x.h, y.h);
    return quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

struct DSConst {
    float rc2;              // cutoff^2 (cell units), compared on the high part
    float rc2_half;         // FP16 phase-1 threshold, as the FP32 kernel
    float rcm;              // sub-cell culling reach
    dsf xi, xi2, c2, selfc; // xi, xi^2, 2 xi / sqrt(pi), 4 xi / sqrt(pi) (cell units)
};

// ---- two double-single pairs at once ---------------------------------------
// The operations above on float2 pairs, one source in flight per lane of the
// FP32x2 arithmetic, each operation rounded once as in the scalar form (a - b
// is fma(b, -1, a)); the cutoff and r = 0 cases become selects (an
// out-of-range source, or a dummy entry, runs on a stand-in r^2 = 1 and
// contributes exactly 0).  Coefficients come from duplicated-pair tables.
__constant__ float2 c_erfcx_ds2_hi[ERFCX_DS_N], c_erfcx_ds2_lo[ERFCX_DS_SPLIT];
__constant__ float2 c_exp_ds2_hi[EXP_DS_N], c_exp_ds2_lo[6];

struct dsf2 {
    float2 h, l;
};
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ dsf2 two_sum2(float2 a, float2 b)
{
    const float2 s = add2(a, b), v = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, v)), sub2(b, v))};
}
__device__ __forceinline__ dsf2 quick_two_sum2(float2 a, float2 b)  // |a| >= |b|
{
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ dsf2 two_prod2(float2 a, float2 b)
{
    const float2 p = mul2(a, b);
    return {p, __ffma2_rn(a, b, neg2(p))};
}
__device__ __forceinline__ dsf2 ds_add2(dsf2 x, dsf2 y)
{
    const dsf2 s = two_sum2(x.h, y.h);
    return quick_two_sum2(s.h, add2(s.l, add2(x.l, y.l)));
}
__device__ __forceinline__ dsf2 ds_add_f2(dsf2 x, float2 y)
{
    const dsf2 s = two_sum2(x.h, y);
    return quick_two_sum2(s.h, add2(s.l, x.l));
}
__device__ __forceinline__ dsf2 ds_mul2(dsf2 x, dsf2 y)
{
    const float2 p = mul2(x.h, y.h);
    const float2 e = __ffma2_rn(x.h, y.l, __ffma2_rn(x.l, y.h, __ffma2_rn(x.h, y.h, neg2(p))));
    return quick_two_sum2(p, e);
}
__device__ __forceinline__ dsf2 dup(dsf c) { return {f2(c.h), f2(c.l)}; }
__device__ __forceinline__ dsf2 sel(bool a, bool b, dsf2 x, dsf2 y)  // lane-wise a, b ? x : y
{
    return {make_float2(a ? x.h.x : y.h.x, b ? x.h.y : y.h.y), make_float2(a ? x.l.x : y.l.x, b ? x.l.y : y.l.y)};
}

// e^{-y} for 0 <= y <= ~60: y = n ln2 - s with |s| <= ln2/2 (ln2 split so that
// n ln2_hi is exact and n ln2_mid is carried exactly by a two-product), e^s by its
// Taylor series to s^13 (terms from s^6 on in FP32: they are below 3e-6), then
// the exact scaling by 2^-n.
__device__ __forceinline__ dsf2 exp_neg_ds2(dsf2 y)
{
    const float kLn2Hi = 0.693145751953125f, kLn2Mid = 1.428606765330187e-06f, kLn2Lo = 5.497923148104107e-14f;
    const float2 n = make_float2(rintf(y.h.x * 1.44269504088896341f), rintf(y.h.y * 1.44269504088896341f));
    const float2 a = __ffma2_rn(n, f2(kLn2Hi), neg2(y.h));
    const dsf2 m = two_prod2(n, f2(kLn2Mid));
    dsf2 s = two_sum2(a, m.h);
    s = quick_two_sum2(s.h, add2(s.l, add2(m.l, __ffma2_rn(n, f2(kLn2Lo), neg2(y.l)))));
    float2 q = c_exp_ds2_hi[EXP_DS_N - 1];
#pragma unroll
    for (int k = EXP_DS_N - 2; k >= 6; --k)
        q = __ffma2_rn(q, s.h, c_exp_ds2_hi[k]);
    dsf2 p = {q, f2(0.f)};
#pragma unroll
    for (int k = 5; k >= 3; --k)
        p = ds_add2(ds_mul2(p, s), {c_exp_ds2_hi[k], c_exp_ds2_lo[k]});
#pragma unroll
    for (int k = 2; k >= 0; --k)
        p = ds_add_f2(ds_mul2(p, s), c_exp_ds2_hi[k]);
    const float2 sc = make_float2(__int_as_float((127 - (int)n.x) << 23), __int_as_float((127 - (int)n.y) << 23));
    return {mul2(p.h, sc), mul2(p.l, sc)};
}

// erfcx(x) = t g(u), t = 1/(1 + x/2), u = (8t - 5)/3 (fit_erf.py: 1.2e-13
// relative on [0, 6]); g's coefficients from k = ERFCX_DS_SPLIT on are below
// 7e-6 and summed in FP32.
__device__ __forceinline__ dsf2 erfcx_ds2(dsf2 x)
{
    const dsf2 den = ds_add_f2({mul2(x.h, f2(0.5f)), mul2(x.l, f2(0.5f))}, f2(1.0f));
    const float2 t0 = make_float2(__frcp_rn(den.h.x), __frcp_rn(den.h.y));
    const dsf2 pr = ds_mul2(den, {t0, f2(0.f)});
    dsf2 t = quick_two_sum2(t0, mul2(t0, sub2(sub2(f2(1.0f), pr.h), pr.l)));
    // past the fit (x > 6): never for an in-range pair
    t = sel(t.h.x < 0.25f, t.h.y < 0.25f, {f2(0.25f), f2(0.f)}, t);
    const dsf2 u = ds_mul2(ds_add_f2({mul2(t.h, f2(8.0f)), mul2(t.l, f2(8.0f))}, f2(-5.0f)),
                           {f2(0.3333333432674408f), f2(-9.934107758624577e-09f)});
    float2 q = c_erfcx_ds2_hi[ERFCX_DS_N - 1];
#pragma unroll
    for (int k = ERFCX_DS_N - 2; k >= ERFCX_DS_SPLIT; --k)
        q = __ffma2_rn(q, u.h, c_erfcx_ds2_hi[k]);
    dsf2 g = {q, f2(0.f)};
#pragma unroll
    for (int k = ERFCX_DS_SPLIT - 1; k >= 0; --k)
        g = ds_add2(ds_mul2(g, u), {c_erfcx_ds2_hi[k], c_erfcx_ds2_lo[k]});
    return ds_mul2(t, g);
}

// Two double-single candidates (cell units): d = (hi diff, exact) + (lo diff)
// per component as (source 0, source 1) pairs, forces fh + fl likewise; adds
// the pairs' terms to the two lanes of acc.
__device__ __forceinline__ void pair_ds2(const float2 (&dh)[3], const float2 (&dl)[3], const float2 (&fh)[3],
                                         const float2 (&fl)[3], const DSConst &k, dsf2 (&acc)[3])
{
    const dsf2 d[3] = {two_sum2(dh[0], dl[0]), two_sum2(dh[1], dl[1]), two_sum2(dh[2], dl[2])};
    const dsf2 r2 = ds_add2(ds_add2(ds_mul2(d[0], d[0]), ds_mul2(d[1], d[1])), ds_mul2(d[2], d[2]));
    // inside the cutoff by the FP32 forms' r^2 (the high parts of d are the FP32
    // kernel's d): with a split near field this pass and the FP32 one divide
    // the pairs at r1 exactly
    const float q0 = pair_r2(d[0].h.x, d[1].h.x, d[2].h.x), q1 = pair_r2(d[0].h.y, d[1].h.y, d[2].h.y);
    const bool in0 = q0 <= k.rc2 && r2.h.x > 0.0f, in1 = q1 <= k.rc2 && r2.h.y > 0.0f;
    const bool z0 = r2.h.x == 0.0f, z1 = r2.h.y == 0.0f;
    const dsf2 r2s = sel(in0, in1, r2, {f2(1.0f), f2(0.f)});
    // 1/r: FP32 estimate and one Newton step carried in double-single
    const float2 y0 = make_float2(rsqrtf(r2s.h.x), rsqrtf(r2s.h.y));
    const dsf2 t = ds_mul2(r2s, two_prod2(y0, y0));
    const dsf2 rinv = quick_two_sum2(y0, mul2(mul2(f2(0.5f), y0), sub2(sub2(f2(1.0f), t.h), t.l)));
    const dsf2 x = ds_mul2(dup(k.xi), ds_mul2(r2s, rinv));
    const dsf2 E = exp_neg_ds2(ds_mul2(dup(k.xi2), r2s));      // e^{-xi^2 r^2}
    const dsf2 A = ds_mul2(ds_mul2(E, erfcx_ds2(x)), rinv);     // erfc(xi r) / r
    const dsf2 B = ds_mul2(dup(k.c2), E);
    const dsf2 zero = {f2(0.f), f2(0.f)};
    const dsf2 nself = {f2(-k.selfc.h), f2(-k.selfc.l)};
    const dsf2 amb = sel(in0, in1, ds_add2(A, {neg2(B.h), neg2(B.l)}), sel(z0, z1, nself, zero));
    const dsf2 apb = ds_add2(A, B);
    const dsf2 f[3] = {{fh[0], fl[0]}, {fh[1], fl[1]}, {fh[2], fl[2]}};
    const dsf2 rf = ds_add2(ds_add2(ds_mul2(d[0], f[0]), ds_mul2(d[1], f[1])), ds_mul2(d[2], f[2]));
    const dsf2 co = sel(in0, in1, ds_mul2(ds_mul2(apb, rf), ds_mul2(rinv, rinv)), zero);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        acc[c] = ds_add2(acc[c], ds_add2(ds_mul2(amb, f[c]), ds_mul2(co, d[c])));
}

// Double-single ring: the FP32 kernel's two 64-source tiles in four groups of
// 33 entries (entry 0 of a group its dummy): sa = (hi + colleague offset,
// lo.x), sb = (lo.y, lo.z, fh.x, fh.y), sc = (fh.z, fl.x, fl.y, fl.z); and per
// slot the FP16 copy of the positions for phase 1.
struct TileDS {
    float4 sa[4 * kGrp];
    float4 sb[4 * kGrp];
    float4 sc[4 * kGrp];
    uint4 sh[2][kT32 / 2];
};
using WsDS = WarpSmem<TileDS>;

// Stage tile `tile` of the warp's stream into ring slot `slot` (as stage_f32,
// with the forces' low parts).
__device__ __forceinline__ void stage_ds(const P2PArgs &a, WsDS &ws, int nseg, int slot, int tile,
                                         int ntile, int total, int lane, int (&sg)[2])
{
    const float4 *rec = (const float4 *)a.nrec, *flo = (const float4 *)a.nflo;
    float3 hp[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h, q = tile + k * ntile;
        if (q < total) {
            if (tile == 0)
                sg[h] = seg_of(ws, nseg, q);
            else if (ws.seg_pref[sg[h] + 1] <= q)
                ++sg[h];
            int dx, dy, dz;
            const int j = seg_element(ws, sg[h], q, dx, dy, dz);
            float3 hi, lo, f;
            unpack_rec(rec[2 * j], rec[2 * j + 1], hi, lo, f);
            const float4 fl = flo[j];
            hp[h] = make_float3(hi.x + (float)dx, hi.y + (float)dy, hi.z + (float)dz);
            const int e = kGrp * (2 * slot + (lane >> 4)) + 1 + (lane & 15) + 16 * h;
            ws.tile.sa[e] = make_float4(hp[h].x, hp[h].y, hp[h].z, lo.x);
            ws.tile.sb[e] = make_float4(lo.y, lo.z, f.x, f.y);
            ws.tile.sc[e] = make_float4(f.z, fl.x, fl.y, fl.z);
        } else {
            hp[h] = make_float3(kFarHalf, kFarHalf, kFarHalf);
        }
    }
    const __half2 hx = __floats2half2_rn(hp[0].x, hp[1].x);
    const __half2 hy = __floats2half2_rn(hp[0].y, hp[1].y);
    const __half2 hz = __floats2half2_rn(hp[0].z, hp[1].z);
    ws.tile.sh[slot][lane] = make_uint4(*(const unsigned *)&hx, *(const unsigned *)&hy,
                                        *(const unsigned *)&hz, 0u);
}

// One work item by one warp: the FP32 kernel's rounds over the ring (the
// busiest lane's count of in-range sources per round, lanes done early going
// on into the next tile), one double-single pair per iteration.
__device__ __forceinline__ bool p2p_ds_run(const P2PArgs &a, const DSConst &kc, int item, WsDS &ws, int lane,
                                           int &t_out, bool &act_out, dsf (&u)[3])
{
    const float4 *rec = (const float4 *)a.nrec;
    int c, tb, te, tsplit;
    if (!find_item(a, item, c, tb, te, tsplit))
        return false;  // past the last real item: the same for the whole warp
    const int t = tb + lane;
    const bool active = t < te;
    t_out = t;
    act_out = active;
    float3 th = make_float3(0.f, 0.f, 0.f), tl = th, fdum;
    if (active) {
        unpack_rec(rec[2 * t], rec[2 * t + 1], th, tl, fdum);
        if (t >= tsplit)  // relative to cell c: the group's second cell (exact)
            th.x += 1.f;
    }
    const float3 blo = make_float3(warp_min(active ? th.x : 1e30f), warp_min(active ? th.y : 1e30f),
                                   warp_min(active ? th.z : 1e30f));
    const float3 bhi = make_float3(warp_max(active ? th.x : -1e30f), warp_max(active ? th.y : -1e30f),
                                   warp_max(active ? th.z : -1e30f));
    const int nseg = build_segments(a, c, ws, lane, blo, bhi, 0.5f, kc.rcm);
    const int total = ws.seg_pref[nseg];
    const int ntile = (total + kT32 - 1) / kT32;
    const __half2 tx = __float2half2_rn(th.x), ty = __float2half2_rn(th.y),
                  tz = __float2half2_rn(th.z), lim = __float2half2_rn(kc.rc2_half);
    if (lane < 4) {  // the groups' dummy sources
        ws.tile.sa[kGrp * lane] = make_float4(1e3f, 1e3f, 1e3f, 0.f);
        ws.tile.sb[kGrp * lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        ws.tile.sc[kGrp * lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int sg[2] = {0, 0};
    for (int tt = 0; tt < 2 && tt < ntile; ++tt)
        stage_ds(a, ws, nseg, tt, tt, ntile, total, lane, sg);
    __syncwarp();
    BitQueue q = {0u, 0u, 0u, 0u, 0};
    if (active) {
        if (ntile > 0)
            phase1_words(ws.tile.sh[0], tx, ty, tz, lim, q.w0, q.w1);
        if (ntile > 1)
            phase1_words(ws.tile.sh[1], tx, ty, tz, lim, q.w2, q.w3);
    }
    // two sources in flight: the lanes of FP32x2 double-single sums
    dsf2 acc[3] = {{f2(0.f), f2(0.f)}, {f2(0.f), f2(0.f)}, {f2(0.f), f2(0.f)}};
    for (int o = 0; o < ntile; ++o) {
        const int need = (int)__reduce_max_sync(0xffffffffu, (unsigned)q.pending());
        for (int it = 0; it < (need + 1) >> 1; ++it) {
            const int e0 = q.pop(), e1 = q.pop();
            const float4 a0 = ws.tile.sa[e0], b0 = ws.tile.sb[e0], c0 = ws.tile.sc[e0];
            const float4 a1 = ws.tile.sa[e1], b1 = ws.tile.sb[e1], c1 = ws.tile.sc[e1];
            const float2 dh[3] = {make_float2(th.x - a0.x, th.x - a1.x), make_float2(th.y - a0.y, th.y - a1.y),
                                  make_float2(th.z - a0.z, th.z - a1.z)};
            const float2 dl[3] = {make_float2(tl.x - a0.w, tl.x - a1.w), make_float2(tl.y - b0.x, tl.y - b1.x),
                                  make_float2(tl.z - b0.y, tl.z - b1.y)};
            const float2 fh[3] = {make_float2(b0.z, b1.z), make_float2(b0.w, b1.w), make_float2(c0.x, c1.x)};
            const float2 fl[3] = {make_float2(c0.y, c1.y), make_float2(c0.z, c1.z), make_float2(c0.w, c1.w)};
            pair_ds2(dh, dl, fh, fl, kc, acc);
        }
        q.shift_if((q.g >> 1) == (o & 1));
        q.shift_if((q.g >> 1) == (o & 1));
        if (o + 2 < ntile) {
            __syncwarp();
            stage_ds(a, ws, nseg, o & 1, o + 2, ntile, total, lane, sg);
            __syncwarp();
            unsigned c0 = 0u, c1 = 0u;
            if (active)
                phase1_words(ws.tile.sh[o & 1], tx, ty, tz, lim, c0, c1);
            const bool odd = q.g & 1;
            q.w1 = odd ? c0 : q.w1;
            q.w2 = odd ? c1 : c0;
            q.w3 = odd ? 0u : c1;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        u[c] = ds_add({acc[c].h.x, acc[c].l.x}, {acc[c].h.y, acc[c].l.y});
    return true;
}

__device__ __forceinline__ void p2p_ds_item(const P2PArgs &a, const DSConst &kc, int item, WsDS &ws,
                                            int lane)
{
    dsf u[3];
    int t;
    bool active;
    if (!p2p_ds_run(a, kc, item, ws, lane, t, active, u))
        return;
    if (active) {
        const int i = a.permn[t];
        double *un = (double *)a.un;
        const double inv_cell = 1.0 / a.cell;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            un[3 * i + c] = ((double)u[c].h + (double)u[c].l) * inv_cell;
    }
}

// Split near field (FP32-bulk plans at tol <= 1e-7): the pairs beyond r1 in
// the compensated FP32 form (their terms are small: e^{-xi^2 r^2} and
// erfc(xi r) decay, so FP32's relative error on them stays below the
// tolerance), those within r1 -- the self term included -- in double-single;
// both passes over the same item in one warp, summed in FP64.
union WsSplit {
    WsF32 f;
    WsDS d;
};

__device__ __forceinline__ void p2p_split_item(const P2PArgs &a, const F32Const &k32, const DSConst &kds,
                                               int item, WsSplit &ws, int lane)
{
    double uo[3];
    dsf ui[3];
    int t;
    bool active;
    if (!p2p_f32_run<true, true>(a, k32, item, ws.f, lane, t, active, uo))
        return;
    __syncwarp();
    p2p_ds_run(a, kds, item, ws.d, lane, t, active, ui);
    if (active) {
        const int i = a.permn[t];
        double *un = (double *)a.un;
        const double inv_cell = 1.0 / a.cell;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            un[3 * i + c] = (((double)ui[c].h + (double)ui[c].l) + uo[c]) * inv_cell;
    }
}

// The warps stride over the work items (the grid holds as many blocks as fit
// at once): the heavier double-single pairs make a partial second wave costly.
__global__ void __launch_bounds__(kWarps * 32) k_p2p_ds(P2PArgs a, DSConst kc, int items)
{
    __shared__ WsDS wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int item = blockIdx.x * kWarps + warp; item < items; item += gridDim.x * kWarps) {
        p2p_ds_item(a, kc, item, wsm[warp], lane);
        __syncwarp();
    }
}

// five blocks an SM (the shared ring allows five; registers fit without spills)
__global__ void __launch_bounds__(kWarps * 32, 5) k_p2p_split(P2PArgs a, F32Const k32, DSConst kds, int items)
{
    __shared__ WsSplit wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int item = blockIdx.x * kWarps + warp; item < items; item += gridDim.x * kWarps) {
        p2p_split_item(a, k32, kds, item, wsm[warp], lane);
        __syncwarp();
    }
}

// ---- double-layer near field in FP32 (Sec. 2.3) ------------------------------
// The Stokeslet kernel's machinery -- cell-group work items, sub-cell culling,
// strided two-tile ring, FP16x2 phase 1, bit queue, two branch-free pairs per
// iteration -- applied to the double-layer term (reading c20):
//   T^N(r) : S = 2 beta (r.S.r) r + 2 gamma (tr S r + 2 S r),
//   beta  = -e^{-x^2} [3 erfcx(x) / r^5 + (2 xi/sqrt(pi)) (3/r^4 + 2 xi^2/r^2)],
//   gamma = (2 xi^3/sqrt(pi)) e^{-x^2},   x = xi r,
// with S the symmetric part of q (x) n of the source (T^F is odd: no self
// term, pairs at r = 0 are skipped).  Cell units throughout (T is homogeneous
// of degree -2, so the sum is scaled by 1/cell^2 at the end).  Source records
// (48 bytes, near order): (lo.x, lo.y, lo.z, S_xx), (S_yy, S_zz, hi bits
// 0..31, hi bits 32..63), (S_xy, S_xz, S_yz, 0); hi and lo as in the
// Stokeslet records.  Ring entries: sa = (hi + colleague offset, lo.x),
// sb = (lo.y, lo.z, S_xx, S_yy), sc = (S_zz, S_xy, S_xz, S_yz).
struct TileDL {
    float4 sa[4 * kGrp];
    float4 sb[4 * kGrp];
    float4 sc[4 * kGrp];
    uint4 sh[2][kT32 / 2];
};
using WsDL = WarpSmem<TileDL>;

struct DLConst {
    float rc2, rc2_half, rcm, xi, nxi2log2e, c2, c2xi2;  // cell units; c2 = 2 xi/sqrt(pi)
};

__device__ __forceinline__ void stage_dl(const P2PArgs &a, const float4 *__restrict__ drec, WsDL &ws, int nseg,
                                         int slot, int tile, int ntile, int total, int lane, int (&sg)[2])
{
    float3 hp[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h, q = tile + k * ntile;
        if (q < total) {
            if (tile == 0)
                sg[h] = seg_of(ws, nseg, q);
            else if (ws.seg_pref[sg[h] + 1] <= q)
                ++sg[h];
            int dx, dy, dz;
            const int j = seg_element(ws, sg[h], q, dx, dy, dz);
            const float4 A = drec[3 * j], B = drec[3 * j + 1], C = drec[3 * j + 2];
            const unsigned w0 = __float_as_uint(B.z), w1 = __float_as_uint(B.w);
            const unsigned qx = w0 & 0x1FFFFFu, qy = (w0 >> 21) | ((w1 & 0x3FFu) << 11), qz = w1 >> 10;
            hp[h] = make_float3((float)(int)qx * (1.f / 1048576.f) + (float)dx,
                                (float)(int)qy * (1.f / 1048576.f) + (float)dy,
                                (float)(int)qz * (1.f / 1048576.f) + (float)dz);
            const int e = kGrp * (2 * slot + (lane >> 4)) + 1 + (lane & 15) + 16 * h;
            ws.tile.sa[e] = make_float4(hp[h].x, hp[h].y, hp[h].z, A.x);
            ws.tile.sb[e] = make_float4(A.y, A.z, A.w, B.x);
            ws.tile.sc[e] = make_float4(B.y, C.x, C.y, C.z);
        } else {
            hp[h] = make_float3(kFarHalf, kFarHalf, kFarHalf);
        }
    }
    const __half2 hx = __floats2half2_rn(hp[0].x, hp[1].x);
    const __half2 hy = __floats2half2_rn(hp[0].y, hp[1].y);
    const __half2 hz = __floats2half2_rn(hp[0].z, hp[1].z);
    ws.tile.sh[slot][lane] = make_uint4(*(const unsigned *)&hx, *(const unsigned *)&hy,
                                        *(const unsigned *)&hz, 0u);
}

// Two double-layer pairs without branches: in range (0 < r^2 <= rc^2) the
// term, else r^2 is replaced by 1e30, for which e^{-x^2}, 1/r^4 and 1/r^5 --
// and with them the term -- are exactly 0.
__device__ __forceinline__ void pair2_dl(const float3 &d0, const float4 &sb0, const float4 &sc0, const float3 &d1,
                                         const float4 &sb1, const float4 &sc1, const DLConst &k, float3 &c0,
                                         float3 &c1)
{
    const float ra = pair_r2(d0.x, d0.y, d0.z), rb = pair_r2(d1.x, d1.y, d1.z);
    const float2 r2s = make_float2(ra <= k.rc2 && ra > 0.f ? ra : 1e30f, rb <= k.rc2 && rb > 0.f ? rb : 1e30f);
    const float2 rinv = make_float2(fast_rsqrt(r2s.x), fast_rsqrt(r2s.y));
    const float2 x = __fmul2_rn(make_float2(k.xi, k.xi), __fmul2_rn(r2s, rinv));
    const float2 ea = __fmul2_rn(r2s, make_float2(k.nxi2log2e, k.nxi2log2e));
    const float2 E = make_float2(fast_ex2(ea.x), fast_ex2(ea.y));
    const float2 den = __ffma2_rn(make_float2((float)ERFCX_C32, (float)ERFCX_C32), x, make_float2(1.f, 1.f));
    const float2 tt = make_float2(fast_rcp(den.x), fast_rcp(den.y));
    float2 p = make_float2(c_erfcx32[ERFCX_F32_N - 1], c_erfcx32[ERFCX_F32_N - 1]);
#pragma unroll
    for (int q = ERFCX_F32_N - 2; q >= 0; --q)
        p = __ffma2_rn(p, tt, make_float2(c_erfcx32[q], c_erfcx32[q]));
    const float2 i2 = __fmul2_rn(rinv, rinv);
    const float2 i4 = __fmul2_rn(i2, i2);
    const float2 i5 = __fmul2_rn(i4, rinv);
    // beta = -E [3 i5 erfcx + c2 (3 i4 + 2 xi^2 i2)]
    const float2 g = __ffma2_rn(make_float2(3.f, 3.f), i4, __fmul2_rn(make_float2(2.f * k.xi * k.xi, 2.f * k.xi * k.xi), i2));
    const float2 in = __ffma2_rn(__fmul2_rn(make_float2(3.f, 3.f), i5), __fmul2_rn(tt, p), __fmul2_rn(make_float2(k.c2, k.c2), g));
    const float2 b2 = __fmul2_rn(make_float2(-2.f, -2.f), __fmul2_rn(E, in));        // 2 beta
    const float2 g2 = __fmul2_rn(make_float2(2.f * k.c2xi2, 2.f * k.c2xi2), E);       // 2 gamma
    // S r, r.S.r, tr S per pair
    const float3 d[2] = {d0, d1};
    const float4 sb[2] = {sb0, sb1}, sc[2] = {sc0, sc1};
    float3 out[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const float Sxx = sb[u].z, Syy = sb[u].w, Szz = sc[u].x, Sxy = sc[u].y, Sxz = sc[u].z, Syz = sc[u].w;
        const float sx = fmaf(Sxx, d[u].x, fmaf(Sxy, d[u].y, Sxz * d[u].z));
        const float sy = fmaf(Sxy, d[u].x, fmaf(Syy, d[u].y, Syz * d[u].z));
        const float sz = fmaf(Sxz, d[u].x, fmaf(Syz, d[u].y, Szz * d[u].z));
        const float rsr = fmaf(sx, d[u].x, fmaf(sy, d[u].y, sz * d[u].z));
        const float tr = Sxx + Syy + Szz;
        const float bb = (u == 0 ? b2.x : b2.y) * rsr, gg = u == 0 ? g2.x : g2.y;
        const float cr = fmaf(gg, tr, bb);  // 2 beta rSr + 2 gamma trS
        const float g4 = 2.f * gg;           // 2 gamma x 2 S r
        out[u] = make_float3(fmaf(cr, d[u].x, g4 * sx), fmaf(cr, d[u].y, g4 * sy), fmaf(cr, d[u].z, g4 * sz));
    }
    c0 = out[0];
    c1 = out[1];
}

// One work item of the double-layer near field by one warp; adds the sums
// (times inv_cell2) into the plan's FP32 near result un, user order, which
// the Stokeslet P2P wrote before it on the same stream.
__device__ __forceinline__ void p2p_dl32_item(const P2PArgs &a, const float4 *__restrict__ drec, const DLConst &kc,
                                              double inv_cell2, float *__restrict__ u, int item, WsDL &ws,
                                              int lane)
{
    int c, tb, te, tsplit;
    if (!find_item(a, item, c, tb, te, tsplit))
        return;
    const int t = tb + lane;
    const bool active = t < te;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
    if (active) {
        const float4 *rec = (const float4 *)a.nrec;
        float3 hi, lo, f;
        unpack_rec(rec[2 * t], rec[2 * t + 1], hi, lo, f);
        th = make_float4(hi.x + (t >= tsplit ? 1.f : 0.f), hi.y, hi.z, 0.f);
        tl = make_float4(lo.x, lo.y, lo.z, 0.f);
    }
    const float3 blo = make_float3(warp_min(active ? th.x : 1e30f), warp_min(active ? th.y : 1e30f),
                                   warp_min(active ? th.z : 1e30f));
    const float3 bhi = make_float3(warp_max(active ? th.x : -1e30f), warp_max(active ? th.y : -1e30f),
                                   warp_max(active ? th.z : -1e30f));
    const int nseg = build_segments(a, c, ws, lane, blo, bhi, 0.5f, kc.rcm);
    const int total = ws.seg_pref[nseg];
    const int ntile = (total + kT32 - 1) / kT32;
    const __half2 tx = __float2half2_rn(th.x), ty = __float2half2_rn(th.y), tz = __float2half2_rn(th.z),
                  lim = __float2half2_rn(kc.rc2_half);
    if (lane < 4) {  // the groups' dummy sources: far away, S = 0
        ws.tile.sa[kGrp * lane] = make_float4(1e3f, 1e3f, 1e3f, 0.f);
        ws.tile.sb[kGrp * lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        ws.tile.sc[kGrp * lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int sg[2] = {0, 0};
    for (int tt = 0; tt < 2 && tt < ntile; ++tt)
        stage_dl(a, drec, ws, nseg, tt, tt, ntile, total, lane, sg);
    __syncwarp();
    BitQueue q = {0u, 0u, 0u, 0u, 0};
    if (active) {
        if (ntile > 0)
            phase1_words(ws.tile.sh[0], tx, ty, tz, lim, q.w0, q.w1);
        if (ntile > 1)
            phase1_words(ws.tile.sh[1], tx, ty, tz, lim, q.w2, q.w3);
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int o = 0; o < ntile; ++o) {
        const int need = (int)__reduce_max_sync(0xffffffffu, (unsigned)q.pending());
        float px = 0.f, py = 0.f, pz = 0.f;
        for (int it = 0; it < (need + 1) >> 1; ++it) {
            const int e0 = q.pop(), e1 = q.pop();
            const float4 s0 = ws.tile.sa[e0], b0 = ws.tile.sb[e0], g0 = ws.tile.sc[e0];
            const float4 s1 = ws.tile.sa[e1], b1 = ws.tile.sb[e1], g1 = ws.tile.sc[e1];
            float3 c0, c1;
            pair2_dl(make_float3((th.x - s0.x) + (tl.x - s0.w), (th.y - s0.y) + (tl.y - b0.x),
                                 (th.z - s0.z) + (tl.z - b0.y)),
                     b0, g0,
                     make_float3((th.x - s1.x) + (tl.x - s1.w), (th.y - s1.y) + (tl.y - b1.x),
                                 (th.z - s1.z) + (tl.z - b1.y)),
                     b1, g1, kc, c0, c1);
            px += c0.x + c1.x;
            py += c0.y + c1.y;
            pz += c0.z + c1.z;
        }
        ux += px;  // per-round FP32 partial sums into FP64 totals
        uy += py;
        uz += pz;
        q.shift_if((q.g >> 1) == (o & 1));
        q.shift_if((q.g >> 1) == (o & 1));
        if (o + 2 < ntile) {
            __syncwarp();
            stage_dl(a, drec, ws, nseg, o & 1, o + 2, ntile, total, lane, sg);
            __syncwarp();
            unsigned c0 = 0u, c1 = 0u;
            if (active)
                phase1_words(ws.tile.sh[o & 1], tx, ty, tz, lim, c0, c1);
            const bool odd = q.g & 1;
            q.w1 = odd ? c0 : q.w1;
            q.w2 = odd ? c1 : c0;
            q.w3 = odd ? 0u : c1;
        }
    }
    if (active) {
        const int i = a.permn[t];
        u[3 * i] = (float)((double)u[3 * i] + ux * inv_cell2);
        u[3 * i + 1] = (float)((double)u[3 * i + 1] + uy * inv_cell2);
        u[3 * i + 2] = (float)((double)u[3 * i + 2] + uz * inv_cell2);
    }
}

__global__ void __launch_bounds__(kWarps * 32) k_p2p_dl32(P2PArgs a, const float4 *__restrict__ drec, DLConst kc,
                                                          double inv_cell2, float *__restrict__ u)
{
    __shared__ WsDL wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    p2p_dl32_item(a, drec, kc, inv_cell2, u, blockIdx.x * kWarps + warp, wsm[warp], lane);
}

// ---- many boxes in one launch ---------------------------------------------
// One persistent launch per P2P variant over the work items of every box of a
// batch: box b owns global items [base[b], base[b + 1]) (its item upper bound,
// cells + N / 32 + 1), a warp finds its box by binary search and runs the
// single-box item code with that box's arguments.  The grid holds as many
// blocks as fit at once; warps stride over the items.
struct BoxP2P {
    P2PArgs a;
    F32Const k32;
    DSConst kds;
    float inv_cell;
    int split;  // double-single plans: 1 for the split near field
};

__device__ __forceinline__ int box_of(const int *base, int nbox, int g)
{
    int lo = 0, hi = nbox;  // base[lo] <= g < base[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// VAR: 0 FP32, 1 FP32 tight (compensated), 2 double-single, 3 FP64
template <int VAR>
__global__ void __launch_bounds__(kWarps * 32) k_p2p_boxes(const BoxP2P *__restrict__ boxes,
                                                           const int *__restrict__ base, int nbox)
{
    using WS = typename std::conditional<
        VAR <= 1, WsF32, typename std::conditional<VAR == 2, WsSplit, WsF64>::type>::type;
    __shared__ WS wsm[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = base[nbox];
    for (int g = blockIdx.x * kWarps + warp; g < total; g += gridDim.x * kWarps) {
        const int b = box_of(base, nbox, g);
        const BoxP2P &bx = boxes[b];
        const int item = g - base[b];
        if constexpr (VAR == 0)
            p2p_f32_item<false>(bx.a, bx.k32, bx.inv_cell, item, wsm[warp], lane);
        else if constexpr (VAR == 1)
            p2p_f32_item<true>(bx.a, bx.k32, bx.inv_cell, item, wsm[warp], lane);
        else if constexpr (VAR == 2) {
            if (bx.split)
                p2p_split_item(bx.a, bx.k32, bx.kds, item, wsm[warp], lane);
            else
                p2p_ds_item(bx.a, bx.kds, item, wsm[warp].d, lane);
        }
        else
            p2p_f64_item(bx.a, item, wsm[warp], lane);
        __syncwarp();
    }
}

bool g_const_loaded[64] = {};

}  // namespace

// Copy the erf/erfcx coefficients into constant memory of the current device
// (once per device).
cudaError_t load_p2p_constants()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_const_loaded[dev])
        return cudaSuccess;
    float c32[ERFCX_F32_N], s32[ERFX_SMALL_N];
    for (int k = 0; k < ERFCX_F32_N; ++k)
        c32[k] = (float)erfcx_f32_c[k];
    for (int k = 0; k < ERFX_SMALL_N; ++k)
        s32[k] = (float)erfx_small_c[k];
    cudaError_t e = cudaMemcpyToSymbol(c_erfcx32, c32, sizeof(c32));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_erfxs32, s32, sizeof(s32));
    if (e == cudaSuccess) {
        float x2[EXP2_F32_N];
        for (int k = 0; k < EXP2_F32_N; ++k)
            x2[k] = (float)exp2_f32_c[k];
        e = cudaMemcpyToSymbol(c_exp2f32, x2, sizeof(x2));
    }
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_erfp64, erf_rat_f64_p, sizeof(erf_rat_f64_p));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_erfq64, erf_rat_f64_q, sizeof(erf_rat_f64_q));
    if (e == cudaSuccess) {  // duplicated pairs for the FP32x2 form
        float2 a[ERFCX_DS_N], b[ERFCX_DS_SPLIT], c[EXP_DS_N], d[6];
        for (int k = 0; k < ERFCX_DS_N; ++k)
            a[k] = make_float2(erfcx_ds_hi[k], erfcx_ds_hi[k]);
        for (int k = 0; k < ERFCX_DS_SPLIT; ++k)
            b[k] = make_float2(erfcx_ds_lo[k], erfcx_ds_lo[k]);
        for (int k = 0; k < EXP_DS_N; ++k)
            c[k] = make_float2(exp_ds_hi[k], exp_ds_hi[k]);
        for (int k = 0; k < 6; ++k)
            d[k] = make_float2(exp_ds_lo[k], exp_ds_lo[k]);
        e = cudaMemcpyToSymbol(c_erfcx_ds2_hi, a, sizeof(a));
        if (e == cudaSuccess)
            e = cudaMemcpyToSymbol(c_erfcx_ds2_lo, b, sizeof(b));
        if (e == cudaSuccess)
            e = cudaMemcpyToSymbol(c_exp_ds2_hi, c, sizeof(c));
        if (e == cudaSuccess)
            e = cudaMemcpyToSymbol(c_exp_ds2_lo, d, sizeof(d));
    }
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        g_const_loaded[dev] = true;
    return e;
}

namespace {

P2PArgs p2p_args(const ewald_plan_s *p)
{
    P2PArgs a;
    a.npos = p->npos;
    a.nfrc = p->nfrc;
    a.nrec = p->nrec;
    a.nflo = p->nflo;
    a.startn = p->startn;
    a.item_off = p->item_off;
    a.permn = p->permn;
    a.un = p->un;
    a.nc = p->g.nc;
    a.K = p->g.K;
    a.ncells = p->g.ncells;
    a.cell = p->g.cell;
    a.rc = p->prm.rc;
    a.xi = p->prm.xi;
    return a;
}

// upper bound on work items: every cell contributes at most count/32 + 1
int64_t p2p_items(const ewald_plan_s *p)
{
    return (int64_t)p->g.ncells + (p->N + kP2PChunk - 1) / kP2PChunk + 1;
}

// the split near field of double-single plans (ds_split_radius): double-single
// pairs within r1 < rc, compensated FP32 beyond
bool p2p_split(const ewald_plan_s *p)
{
    return p->near_ds && p->ds_r1 < p->prm.rc;
}

// cell units: lengths / cell, xi * cell
F32Const f32_const(const ewald_plan_s *p)
{
    F32Const kc;
    const double r1c = p->ds_r1 / p->g.cell;
    kc.r1sq = p2p_split(p) ? (float)(r1c * r1c) : -1.0f;
    const double rcc = p->prm.rc / p->g.cell, xic = p->prm.xi * p->g.cell;
    kc.rc2 = (float)(rcc * rcc);
    kc.rc2_half = half_threshold(rcc);
    kc.rcm = (float)(rcc + 1e-3);  // sub-cell culling reach: |lo| <= 2^-21 fits the margin
    kc.xi = (float)xic;
    const double c = -xic * xic * 1.4426950408889634;  // -xi^2 log2(e), cell units
    kc.nxi2log2e = (float)c;
    kc.nxi2log2e_lo = (float)(c - (double)kc.nxi2log2e);
    kc.c2 = (float)(2.0 * xic / sqrt(3.14159265358979323846));
    kc.selfc = (float)(4.0 * xic / sqrt(3.14159265358979323846));
    return kc;
}

// cell units, every constant as a double-single pair
DSConst ds_const(const ewald_plan_s *p)
{
    auto split = [](double v) {
        dsf r;
        r.h = (float)v;
        r.l = (float)(v - (double)r.h);
        return r;
    };
    DSConst kc;
    // the double-single pass reaches r1 when the near field is split
    const double rcc = (p2p_split(p) ? p->ds_r1 : p->prm.rc) / p->g.cell, xic = p->prm.xi * p->g.cell;
    kc.rc2 = (float)(rcc * rcc);
    kc.rc2_half = half_threshold(rcc);
    kc.rcm = (float)(rcc + 1e-3);
    kc.xi = split(xic);
    kc.xi2 = split(xic * xic);
    kc.c2 = split(2.0 * xic / sqrt(3.14159265358979323846));
    kc.selfc = split(4.0 * xic / sqrt(3.14159265358979323846));
    return kc;
}

// 0 FP32, 1 FP32 tight (compensated sums below tol 1e-6), 2 double-single, 3 FP64
int p2p_variant(const ewald_plan_s *p)
{
    if (p->near_ds)
        return 2;
    if (p->near64)
        return 3;
    return p->prm.tol < 1e-6 ? 1 : 0;
}

unsigned resident_blocks(const void *kernel, int dev)
{
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kWarps * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    return (unsigned)std::max(1, sms * std::max(1, per));
}

}  // namespace

cudaError_t launch_p2p(ewald_plan_s *p, cudaStream_t s)
{
    cudaError_t e = load_p2p_constants();
    if (e != cudaSuccess)
        return e;
    const P2PArgs a = p2p_args(p);
    const int64_t items = p2p_items(p);
    const unsigned grid = (unsigned)((items + kWarps - 1) / kWarps);
    switch (p2p_variant(p)) {
    case 2: {
        int dev = 0;
        cudaGetDevice(&dev);
        if (p2p_split(p)) {
            const unsigned cap = resident_blocks((const void *)k_p2p_split, dev);
            k_p2p_split<<<std::min(grid, cap), kWarps * 32, 0, s>>>(a, f32_const(p), ds_const(p), (int)items);
        } else {
            const unsigned cap = resident_blocks((const void *)k_p2p_ds, dev);
            k_p2p_ds<<<std::min(grid, cap), kWarps * 32, 0, s>>>(a, ds_const(p), (int)items);
        }
        break;
    }
    case 3:
        k_p2p_f64<<<grid, kWarps * 32, 0, s>>>(a);
        break;
    case 1:
        k_p2p_f32<true><<<grid, kWarps * 32, 0, s>>>(a, f32_const(p), (float)(1.0 / p->g.cell));
        break;
    default:
        // four-warp blocks: one-warp blocks spread a single-wave launch more
        // evenly (P2P alone 8 % faster) but leave the concurrent far field
        // less room (measured apply 0.727 against 0.710 ms)
        k_p2p_f32<false><<<grid, kWarps * 32, 0, s>>>(a, f32_const(p), (float)(1.0 / p->g.cell));
    }
    return cudaGetLastError();
}

// Double-layer near field of an FP32 plan (records from build_dl_records),
// added into u (user order).
cudaError_t launch_p2p_dl32(ewald_plan_s *p, const void *drec, cudaStream_t s)
{
    cudaError_t e = load_p2p_constants();
    if (e != cudaSuccess)
        return e;
    const P2PArgs a = p2p_args(p);
    const double rcc = p->prm.rc / p->g.cell, xic = p->prm.xi * p->g.cell;
    DLConst kc;
    kc.rc2 = (float)(rcc * rcc);
    kc.rc2_half = half_threshold(rcc);
    kc.rcm = (float)(rcc + 1e-3);
    kc.xi = (float)xic;
    kc.nxi2log2e = (float)(-xic * xic * 1.4426950408889634);
    kc.c2 = (float)(2.0 * xic / sqrt(3.14159265358979323846));
    kc.c2xi2 = (float)(2.0 * xic * xic * xic / sqrt(3.14159265358979323846));
    const int64_t items = p2p_items(p);
    const unsigned grid = (unsigned)((items + kWarps - 1) / kWarps);
    k_p2p_dl32<<<grid, kWarps * 32, 0, s>>>(a, (const float4 *)drec, kc, 1.0 / (p->g.cell * p->g.cell),
                                            (float *)p->un);
    return cudaGetLastError();
}

// ---- the near field of many plans in one launch per variant ---------------
struct P2PBoxes {
    int dev = 0;
    BoxP2P *boxes[4] = {};  // device, per variant
    int *base[4] = {};      // device, per variant: nbox + 1 prefix offsets of items
    int nbox[4] = {};
    unsigned grid[4] = {};
};

cudaError_t p2p_boxes_create(ewald_plan_s *const *plans, int n, P2PBoxes **out)
{
    cudaError_t e = load_p2p_constants();
    if (e != cudaSuccess)
        return e;
    P2PBoxes *b = new (std::nothrow) P2PBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    cudaGetDevice(&b->dev);
    std::vector<BoxP2P> hb[4];
    std::vector<int> hbase[4];
    for (int v = 0; v < 4; ++v)
        hbase[v].push_back(0);
    for (int i = 0; i < n; ++i) {
        const ewald_plan_s *p = plans[i];
        const int v = p2p_variant(p);
        BoxP2P x;
        x.a = p2p_args(p);
        x.k32 = f32_const(p);
        x.split = p2p_split(p) ? 1 : 0;
        if (v == 2)
            x.kds = ds_const(p);
        x.inv_cell = (float)(1.0 / p->g.cell);
        hb[v].push_back(x);
        hbase[v].push_back(hbase[v].back() + (int)p2p_items(p));
    }
    const void *kern[4] = {(const void *)k_p2p_boxes<0>, (const void *)k_p2p_boxes<1>,
                           (const void *)k_p2p_boxes<2>, (const void *)k_p2p_boxes<3>};
    for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
        b->nbox[v] = (int)hb[v].size();
        if (!b->nbox[v])
            continue;
        e = cudaMalloc(&b->boxes[v], sizeof(BoxP2P) * hb[v].size());
        if (e == cudaSuccess)
            e = cudaMalloc(&b->base[v], sizeof(int) * hbase[v].size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->boxes[v], hb[v].data(), sizeof(BoxP2P) * hb[v].size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->base[v], hbase[v].data(), sizeof(int) * hbase[v].size(), cudaMemcpyHostToDevice);
        const unsigned need = (unsigned)((hbase[v].back() + kWarps - 1) / kWarps);
        b->grid[v] = std::min(need, resident_blocks(kern[v], b->dev));
    }
    if (e != cudaSuccess) {
        p2p_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t p2p_boxes_launch(const P2PBoxes *b, cudaStream_t s)
{
    if (b->nbox[0])
        k_p2p_boxes<0><<<b->grid[0], kWarps * 32, 0, s>>>(b->boxes[0], b->base[0], b->nbox[0]);
    if (b->nbox[1])
        k_p2p_boxes<1><<<b->grid[1], kWarps * 32, 0, s>>>(b->boxes[1], b->base[1], b->nbox[1]);
    if (b->nbox[2])
        k_p2p_boxes<2><<<b->grid[2], kWarps * 32, 0, s>>>(b->boxes[2], b->base[2], b->nbox[2]);
    if (b->nbox[3])
        k_p2p_boxes<3><<<b->grid[3], kWarps * 32, 0, s>>>(b->boxes[3], b->base[3], b->nbox[3]);
    return cudaGetLastError();
}

int p2p_boxes_launches(const P2PBoxes *b)
{
    int k = 0;
    for (int v = 0; v < 4; ++v)
        k += b->nbox[v] ? 1 : 0;
    return k;
}

void p2p_boxes_destroy(P2PBoxes *b)
{
    if (!b)
        return;
    for (int v = 0; v < 4; ++v) {
        if (b->boxes[v])
            cudaFree(b->boxes[v]);
        if (b->base[v])
            cudaFree(b->base[v]);
    }
    delete b;
}

}  // namespace ewg
