// k_grid_ds.cu -- steps a2 (P2G, eq. (p2g)) and a6 (G2P, eq. (g2p)) in
// double-single arithmetic, for the FP32-bulk plans at tol <= 1e-7 (whose near
// field is double-single too): on this GPU the FP64 pipe runs at a small
// fraction of the FP32 one, and FP64 grid kernels were most of such an apply.
//
// A double-single value is h + l, two FP32 numbers (~44 significant bits).
// Product x y: p = x.h y.h and its error term e = fma(x.h, y.h, -p) + x.h y.l
// + x.l y.h (x.l y.l lies below 2^-44 relative), left unnormalised.  Sum
// a += p + e: Knuth's two-sum of a.h + p, whose rounding error goes into a.l
// together with e.  a.l is never renormalised: it stays within a few ulp of the
// largest partial sum, so a.h + a.l carries ~2^-44 of it.  The _rn intrinsics
// keep the compiler from contracting the products into the sums.
//
// Window weights (Sec. 2.2, Sec. 4): evaluated once per binning for every
// point by FP64 Horner on the window polynomial and stored split h + l, the P
// bins of an axis padded to PW (a multiple of 4).  P2G reads them for every
// tile a point touches, G2P once per point.
//
// P2G: owner-computes over tiles of 8^3 grid points, as the FP32 kernel of
// k_grid.cu, with one thread per (y, z) row of the tile holding the row's 8 x 3
// double-single sums.  A warp holds the 32 rows of one z-half, so the z-halves
// and x-halves a point's support misses are skipped warp-uniformly.  The sums
// are rounded to FP64 on the store (cuFFT's input).
//
// G2P: from a double-single copy of the FP64 grid (h = fl32(v), l = fl32(v -
// h)), staged per tile and component in shared memory (below).
#include <cuda.h>  // CUtensorMap (the type; descriptors are encoded by k_grid.cu's helper)
#include <string.h>

#include <map>
#include <new>
#include <vector>

#include "internal.h"

namespace ewg {
namespace {

__device__ __forceinline__ void ds_prod(float xh, float xl, float yh, float yl, float &p, float &e)
{
    p = __fmul_rn(xh, yh);
    e = fmaf(xl, yh, fmaf(xh, yl, fmaf(xh, yh, -p)));
}

// (ah, al) += p + e
__device__ __forceinline__ void ds_acc(float &ah, float &al, float p, float e)
{
    const float s = __fadd_rn(ah, p);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    ah = s;
    al = __fadd_rn(al, __fadd_rn(err, e));
}

// (ah, al) += x y
__device__ __forceinline__ void ds_fma(float &ah, float &al, float xh, float xl, float yh, float yl)
{
    float p, e;
    ds_prod(xh, xl, yh, yl, p, e);
    ds_acc(ah, al, p, e);
}

// ds_fma on two sums at once in FP32x2 arithmetic: (ah, al) += (xh, xl) y,
// y = (yh, yl) common to both lanes and passed negated (nyh = -yh, nyl = -yl).
// The same operations, each rounded once: a - b is fma(b, -1, a).
__device__ __forceinline__ void ds_fma2(float2 &ah, float2 &al, float2 xh, float2 xl, float2 yh, float2 nyh,
                                        float2 nyl)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 p = __fmul2_rn(xh, yh);
    // -(product error + cross terms), exact up to the last two roundings
    const float2 ne = __ffma2_rn(xl, nyh, __ffma2_rn(xh, nyl, __ffma2_rn(xh, nyh, p)));
    const float2 s = __fadd2_rn(ah, p);
    const float2 bb = __ffma2_rn(ah, m1, s);
    const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, s), m1, ah), __ffma2_rn(bb, m1, p));
    ah = s;
    al = __fadd2_rn(al, __ffma2_rn(ne, m1, err));
}

// ds_fma on two sums at once, both operands per lane: (ah, al) += (xh, xl) (yh, yl)
__device__ __forceinline__ void ds_fma2v(float2 &ah, float2 &al, float2 xh, float2 xl, float2 yh, float2 yl)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 p = __fmul2_rn(xh, yh);
    const float2 e = __ffma2_rn(xl, yh, __ffma2_rn(xh, yl, __ffma2_rn(xh, yh, __fmul2_rn(p, m1))));
    const float2 s = __fadd2_rn(ah, p);
    const float2 bb = __ffma2_rn(ah, m1, s);
    const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, s), m1, ah), __ffma2_rn(bb, m1, p));
    ah = s;
    al = __fadd2_rn(al, __fadd2_rn(err, e));
}

__device__ __forceinline__ void ds_split(double v, float &h, float &l)
{
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

__device__ __forceinline__ double ds_join(float h, float l) { return (double)h + (double)l; }

struct GridDsArgs {
    const dvec4 *tdat;       // tile-sorted (delta, packed anchor offsets)
    const float4 *tfrc;      // tile-sorted forces: [2 p] = h, [2 p + 1] = l (w unused)
    const float *wts;        // window weights [p][axis][h: PW | l: PW]
    const int32_t *startt, *permt;
    int P, PW, M, nt, KT;
    double *grid;            // P2G output, 3 M^3 FP64
    const float *gds;        // G2P input: 3 M^3 h values, then 3 M^3 l values
    double *uf;              // G2P output, user order
    double scale;            // G2P: multiplies the sum
};

// ---- window weights ---------------------------------------------------------
__device__ __forceinline__ void window_ds_body(const dvec4 *__restrict__ tdat, const double *__restrict__ coef,
                                               float *__restrict__ wts, int64_t N, int P, int deg, int PW,
                                               int64_t q)  // (point, axis)
{
    if (q >= 3 * N)
        return;
    const int64_t p = q / 3;
    const int d = (int)(q - 3 * p);
    const dvec4 td = tdat[p];
    const double z = 2.0 * (d == 0 ? td.x : (d == 1 ? td.y : td.z)) - 1.0;
    float *w = wts + q * 2 * PW;
    const int nd = deg + 1;
    // bins j and P-1-j from bin j's polynomial: the window is even, so bin
    // P-1-j at z is bin j at -z, E(z^2) -+ z O(z^2) with E, O its even and
    // odd parts (half the FP64 Horner work)
    const double z2 = z * z;
    const int ke = deg & ~1, ko = (deg & 1) ? deg : deg - 1;  // top even and odd powers
    for (int j = 0; j < (P + 1) / 2; ++j) {
        const double *c = coef + j * nd;
        double e = c[ke], o = ko >= 1 ? c[ko] : 0.0;
        for (int k = ke - 2; k >= 0; k -= 2)
            e = fma(e, z2, c[k]);
        for (int k = ko - 2; k >= 1; k -= 2)
            o = fma(o, z2, c[k]);
        float h, l;
        ds_split(fma(z, o, e), h, l);
        w[j] = h;
        w[PW + j] = l;
        if (P - 1 - j != j) {
            ds_split(fma(-z, o, e), h, l);
            w[P - 1 - j] = h;
            w[PW + P - 1 - j] = l;
        }
    }
    for (int j = P; j < PW; ++j) {
        w[j] = 0.f;
        w[PW + j] = 0.f;
    }
}

__global__ void k_window_ds(const dvec4 *__restrict__ tdat, const double *__restrict__ coef,
                            float *__restrict__ wts, int64_t N, int P, int deg, int PW)
{
    window_ds_body(tdat, coef, wts, N, P, deg, PW, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// many boxes' window weights and double-single grid copies in one launch each
struct WindowJob {
    const dvec4 *tdat;
    const double *coef;
    float *wts;
    int64_t N;
    int P, deg, PW;
};
__global__ void k_window_ds_jobs(const WindowJob *__restrict__ jobs, const int *__restrict__ base, int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const WindowJob &j = jobs[b];
    window_ds_body(j.tdat, j.coef, j.wts, j.N, j.P, j.deg, j.PW,
                   (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x);
}
struct SplitJob {
    const double *src;
    float *dst;
    int64_t n;
};
__global__ void k_grid_split_jobs(const SplitJob *__restrict__ jobs, const int *__restrict__ base, int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const SplitJob &j = jobs[b];
    const int64_t i = (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x;
    if (i >= j.n)
        return;
    float h, l;
    ds_split(j.src[i], h, l);
    j.dst[i] = h;
    j.dst[j.n + i] = l;
}

// ---- P2G --------------------------------------------------------------------
constexpr int kT = 8, kH = 4;
constexpr int kP2GDsThreads = 256;
constexpr int kDsRows = kT * kT;                      // one thread per (y, z) row
constexpr int kDsSlices = kP2GDsThreads / kDsRows;    // point slices
constexpr int kDsMaxSeg = 27;                         // (KT + 1)^3, KT = ceil((P-1)/8) <= 2

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

template <int PC>
__device__ __forceinline__ void p2g_ds_body(const GridDsArgs &a, const int tile)
{
    constexpr int NT = kP2GDsThreads, B = NT, T = kT, H = kH, SL = kDsSlices, T3 = T * T * T;
    extern __shared__ __align__(16) unsigned char smem[];
    float *wr = (float *)smem;                  // [6][B][T] rows: x h, x l, y h, y l, z h, z l
    float4 *sf = (float4 *)(wr + 6 * B * T);    // [B][2] force h, l
    __shared__ int soff[B], sidx[B];
    __shared__ int seg_start[kDsMaxSeg], seg_pref[kDsMaxSeg + 1];
    __shared__ int scount;

    const int nt = a.nt, KT = a.KT, side = KT + 1, nseg = side * side * side;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    // the neighbour tiles (dz, dy, dx) in [-KT, 0]^3 whose anchors can reach
    // this tile: their point ranges, concatenated
    if (threadIdx.x < 32) {
        const int s = threadIdx.x;
        int len = 0;
        if (s < nseg) {
            const int dx = s % side - KT, dy = (s / side) % side - KT, dz = s / (side * side) - KT;
            const int nb = (wrapi(tz + dz, nt) * nt + wrapi(ty + dy, nt)) * nt + wrapi(tx + dx, nt);
            seg_start[s] = a.startt[nb];
            len = a.startt[nb + 1] - a.startt[nb];
        }
        int v = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (s >= o)
                v += u;
        }
        if (s < nseg)
            seg_pref[s + 1] = v;
        if (s == 0)
            seg_pref[0] = 0;
    }
    const int row = threadIdx.x % kDsRows, slice = threadIdx.x / kDsRows;
    const int y = row % T, z = row / T;
    const bool zlo = z < H;  // warp-uniform
    float2 ah[T / 2][3], al[T / 2][3];  // x and x + 1 packed for FP32x2 arithmetic
#pragma unroll
    for (int x = 0; x < T / 2; ++x)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            ah[x][c] = al[x][c] = make_float2(0.f, 0.f);
    __syncthreads();
    const int total = seg_pref[nseg];

    for (int base = 0; base < total; base += B) {
        if (threadIdx.x == 0)
            scount = 0;
        __syncthreads();
        // (A) one thread per candidate: does its support reach the tile?
        const int q = base + threadIdx.x;
        bool keep = false;
        int j = 0, ox = 0, oy = 0, oz = 0;
        if (q < total) {
            int lo = 0, hi = nseg;  // seg_pref[lo] <= q < seg_pref[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (seg_pref[mid] <= q)
                    lo = mid;
                else
                    hi = mid;
            }
            const int s = lo;
            j = seg_start[s] + (q - seg_pref[s]);
            const int dx = s % side - KT, dy = (s / side) % side - KT, dz = s / (side * side) - KT;
            const int packed = (int)a.tdat[j].w;
            ox = dx * T + (packed & 15);
            oy = dy * T + ((packed >> 4) & 15);
            oz = dz * T + ((packed >> 8) & 15);
            keep = ox + PC > 0 && ox < T && oy + PC > 0 && oy < T && oz + PC > 0 && oz < T;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        int wbase = 0;
        if ((threadIdx.x & 31) == 0 && ball)
            wbase = atomicAdd(&scount, __popc(ball));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (keep) {
            const int k = wbase + __popc(ball & ((1u << (threadIdx.x & 31)) - 1u));
            // offsets lie in (-P, T): bias by 32 into 6-bit fields
            soff[k] = (ox + 32) | ((oy + 32) << 6) | ((oz + 32) << 12);
            sidx[k] = j;
        }
        __syncthreads();
        const int n = scount;
        // (B) one thread per (point, axis): the axis' weights on the tile's 8
        // grid lines (zero off the support), h and l rows; and the force
        for (int w = threadIdx.x; w < 3 * n; w += NT) {
            const int k = w / 3, d = w - 3 * k;
            const int o = ((soff[k] >> (6 * d)) & 63) - 32;
            const int jj = sidx[k];
            const float *src = a.wts + ((int64_t)jj * 3 + d) * 2 * a.PW;
            float hv[T], lv[T];
#pragma unroll
            for (int x = 0; x < T; ++x) {
                const int l = x - o;
                const bool in = l >= 0 && l < PC;
                const int li = in ? l : 0;
                hv[x] = in ? __ldg(src + li) : 0.f;
                lv[x] = in ? __ldg(src + a.PW + li) : 0.f;
            }
            float4 *dh = (float4 *)(wr + ((2 * d) * B + k) * T);
            float4 *dl = (float4 *)(wr + ((2 * d + 1) * B + k) * T);
            dh[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
            dh[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
            dl[0] = make_float4(lv[0], lv[1], lv[2], lv[3]);
            dl[1] = make_float4(lv[4], lv[5], lv[6], lv[7]);
            if (d == 0) {
                sf[2 * k] = a.tfrc[2 * (int64_t)jj];
                sf[2 * k + 1] = a.tfrc[2 * (int64_t)jj + 1];
            }
        }
        __syncthreads();
        // (C) the slice's points into this thread's row
        for (int k = slice; k < n; k += SL) {
            const int so = soff[k];
            const int okx = (so & 63) - 32, okz = ((so >> 12) & 63) - 32;
            if (zlo ? okz >= H : okz + PC <= H)
                continue;  // the warp's z-half is off the support
            const bool hx0 = okx < H, hx1 = okx + PC > H;
            float gp, ge;  // wy wz
            ds_prod(wr[(2 * B + k) * T + y], wr[(3 * B + k) * T + y], wr[(4 * B + k) * T + z],
                    wr[(5 * B + k) * T + z], gp, ge);
            const float4 fh = sf[2 * k], fl = sf[2 * k + 1];
            float g[3][2];  // wy wz f
            ds_prod(gp, ge, fh.x, fl.x, g[0][0], g[0][1]);
            ds_prod(gp, ge, fh.y, fl.y, g[1][0], g[1][1]);
            ds_prod(gp, ge, fh.z, fl.z, g[2][0], g[2][1]);
            const float2 *wxh = (const float2 *)(wr + (0 * B + k) * T),
                         *wxl = (const float2 *)(wr + (1 * B + k) * T);
            float2 gh[3], ngh[3], ngl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gh[c] = make_float2(g[c][0], g[c][0]);
                ngh[c] = make_float2(-g[c][0], -g[c][0]);
                ngl[c] = make_float2(-g[c][1], -g[c][1]);
            }
#pragma unroll
            for (int x = 0; x < T / 2; ++x) {
                if (x < H / 2 ? hx0 : hx1) {
                    const float2 h = wxh[x], l = wxl[x];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        ds_fma2(ah[x][c], al[x][c], h, l, gh[c], ngh[c], ngl[c]);
                }
            }
        }
        __syncthreads();
    }
    // sum the slices (reusing the staging area) and store the tile in FP64;
    // [SL][3][T^2][T + 1]: rows padded by one value, so the 32 rows a warp
    // writes at one x spread over the banks (unpadded: 16 rows a bank pair)
    constexpr int RS = T + 1, T3P = T * T * RS;
    float2 *red = (float2 *)smem;
#pragma unroll
    for (int x = 0; x < T; ++x)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            red[(slice * 3 + c) * T3P + (z * T + y) * RS + x] =
                x & 1 ? make_float2(ah[x / 2][c].y, al[x / 2][c].y) : make_float2(ah[x / 2][c].x, al[x / 2][c].x);
    __syncthreads();
    const int M = a.M;
    const int64_t M3 = (int64_t)M * M * M;
    for (int o = threadIdx.x; o < 3 * T3; o += NT) {
        const int c = o / T3, r = o - c * T3;
        float sh = 0.f, sl = 0.f;
#pragma unroll
        const int x = r % T, yy = (r / T) % T, zz = r / (T * T);
#pragma unroll
        for (int qq = 0; qq < SL; ++qq) {
            const float2 v = red[(qq * 3 + c) * T3P + (zz * T + yy) * RS + x];
            ds_acc(sh, sl, v.x, v.y);
        }
        const int64_t gx = tx * T + x, gy = ty * T + yy, gz = tz * T + zz;
        a.grid[c * M3 + (gz * M + gy) * M + gx] = ds_join(sh, sl);
    }
}

constexpr size_t kP2GDsStage = sizeof(float) * 6 * kP2GDsThreads * kT + sizeof(float4) * 2 * kP2GDsThreads;
constexpr size_t kP2GDsRed = sizeof(float2) * kDsSlices * 3 * kT * kT * (kT + 1);
constexpr size_t kP2GDsSmem = kP2GDsStage > kP2GDsRed ? kP2GDsStage : kP2GDsRed;

// ---- G2P --------------------------------------------------------------------
// One block per tile of anchors, one pass per component: the block stages the
// component's (T + P - 1)^3 h and l values its points can touch (16-byte
// asynchronous copies into rows of stride S; M a multiple of 8 keeps every
// 4-float chunk on one side of the periodic wrap, M >= P keeps one wrap
// enough), then one warp per point sums its support: lanes over the P x P
// (y, x) pairs, dealt by bank (g2p_rounds), each walking its z column with
// immediate offsets, s = sum_z wz v, then u += wy wx s.
constexpr int kG2PDsThreads = 256;

template <int PC>
struct G2PDs {
    static constexpr int T = kT, RR = T + PC - 1, S = g2p_stride(PC), NR = g2p_rounds(PC, S);
    static constexpr int NCH = (RR + 3) / 4;  // 16-byte chunks per staged row
    static constexpr int PLANE = RR * S, VOL = RR * PLANE;
    static constexpr int VOLP = (VOL + 31) & ~31;  // the l block starts on a 128-byte boundary
    static constexpr int NW = kG2PDsThreads / 32;
    // h and l blocks, per-warp weights, the dealt pairs, the TMA mbarrier, and
    // 128 bytes for aligning the h block
    static constexpr size_t smem =
        sizeof(float) * (2 * (size_t)VOLP + NW * 6 * 16) + sizeof(int) * NR * 32 + 8 + 128;
};

template <int PC>
__device__ __forceinline__ void g2p_ds_body(const GridDsArgs &a, const int tile, const CUtensorMap *tm,
                                            int use_tma, int *err)
{
    using G = G2PDs<PC>;
    constexpr int T = G::T, RR = G::RR, S = G::S, NR = G::NR, NCH = G::NCH, PLANE = G::PLANE,
                  VOLP = G::VOLP, NW = G::NW;
    const int s0 = a.startt[tile], s1 = a.startt[tile + 1];
    if (s0 == s1)
        return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem =
        smem_raw + ((128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
    float *vh = (float *)smem;       // [RR][RR][S] h values of the component
    float *vl = vh + VOLP;           // l values
    float *wsm = vl + VOLP;          // per warp [6][16]: x h, x l, y h, y l, z h, z l
    int *tab = (int *)(wsm + NW * 6 * 16);  // [NR][32] bank-dealt pairs
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(tab + NR * 32);  // 8-byte aligned: 128-byte rows
    const int nt = a.nt, M = a.M, PW = a.PW;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int r = 0;
        for (int yy = 0; yy < PC; ++yy) {
            const int xx = (lane - S * yy) & 31;
            if (xx < PC)
                tab[r++ * 32 + lane] = (yy << 8) | xx;
        }
        for (; r < NR; ++r)
            tab[r * 32 + lane] = -1;
    }
    const int64_t M2 = (int64_t)M * M, M3 = M2 * M;
    const unsigned vh_a = (unsigned)__cvta_generic_to_shared(vh);
    float *w = wsm + warp * 6 * 16;
    // Interior tiles: each component's h and l blocks come by two TMA tensor
    // copies (boxes of S x RR x RR floats of the [6][M][M][M] double-single
    // grid, the staged layout itself), completing phase c of one mbarrier;
    // blocks that wrap around the periodic grid use 16-byte asynchronous copies.
    const bool tma = use_tma && tx * T + S <= M && ty * T + RR <= M && tz * T + RR <= M;
    if (tma) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    for (int c = 0; c < 3; ++c) {
        bool staged = true;
        if (tma) {
            if (threadIdx.x == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                             "r"((unsigned)(2 * sizeof(float) * G::VOL))
                             : "memory");
#pragma unroll
                for (int half = 0; half < 2; ++half)
                    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(vh_a + 4 * half * VOLP),
                                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(tx * T), "r"(ty * T), "r"(tz * T),
                                 "r"(c + 3 * half), "r"(bar_a)
                                 : "memory");
            }
            for (int it = 0, done = 0; !done; ++it) {  // phase c of the barrier, bounded
                unsigned ok;
                asm volatile("{\n\t.reg .pred p;\n\t"
                             "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, p;\n\t}"
                             : "=r"(ok)
                             : "r"(bar_a), "r"(c & 1)
                             : "memory");
                done = ok || it >= (1 << 20);
                staged = ok;
            }
        } else {
            // stage component c: threads over (plane h/l, z, y, chunk)
            const float *srch = a.gds + c * M3, *srcl = a.gds + (3 + c) * M3;
            for (int t = threadIdx.x; t < 2 * RR * RR * NCH; t += kG2PDsThreads) {
                const int half = t / (RR * RR * NCH), r = t - half * (RR * RR * NCH);
                const int row = r / NCH, ch = r - row * NCH;
                const int z = row / RR, y = row - z * RR;
                int gx = tx * T + 4 * ch, gy = ty * T + y, gz = tz * T + z;
                gx -= gx >= M ? M : 0;
                gy -= gy >= M ? M : 0;
                gz -= gz >= M ? M : 0;
                const float *src = (half ? srcl : srch) + (gz * M2 + (int64_t)gy * M + gx);
                const unsigned dst = vh_a + 4 * (half * VOLP + row * S + 4 * ch);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
            }
            asm volatile("cp.async.commit_group;\n" ::);
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (!__syncthreads_and(staged)) {  // the copies did not land: report and leave the tile
            if (threadIdx.x == 0)
                atomicOr(err, 2);
            return;
        }
        // this lane's pairs
        int roff[NR], ry[NR], rx[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int e = tab[r * 32 + lane];
            roff[r] = e >= 0 ? (e >> 8) * S + (e & 255) : -1;
            ry[r] = e >= 0 ? e >> 8 : 0;
            rx[r] = e >= 0 ? e & 255 : 0;
        }
        for (int p = s0 + warp; p < s1; p += NW) {
            const int packed = (int)a.tdat[p].w;
            const int ox = packed & 15, oy = (packed >> 4) & 15, oz = (packed >> 8) & 15;
            const float *wp = a.wts + (int64_t)p * 6 * PW;
            __syncwarp();
            for (int q = lane; q < 6 * PC; q += 32) {
                const int d = q / PC, l = q - d * PC;
                w[d * 16 + l] = __ldg(wp + d * PW + l);
            }
            __syncwarp();
            float wzh[PC], wzl[PC];
#pragma unroll
            for (int k = 0; k < PC; ++k) {
                wzh[k] = w[4 * 16 + k];
                wzl[k] = w[5 * 16 + k];
            }
            const int base = (oz * RR + oy) * S + ox;
            float uh = 0.f, ul = 0.f;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (roff[r] >= 0) {
                    const float *ch = vh + base + roff[r], *cl = vl + base + roff[r];
                    // even and odd planes as the two lanes of FP32x2 sums
                    float2 sh2 = make_float2(0.f, 0.f), sl2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k + 1 < PC; k += 2)
                        ds_fma2v(sh2, sl2, make_float2(wzh[k], wzh[k + 1]), make_float2(wzl[k], wzl[k + 1]),
                                 make_float2(ch[k * PLANE], ch[(k + 1) * PLANE]),
                                 make_float2(cl[k * PLANE], cl[(k + 1) * PLANE]));
                    if constexpr (PC % 2)
                        ds_fma(sh2.x, sl2.x, wzh[PC - 1], wzl[PC - 1], ch[(PC - 1) * PLANE], cl[(PC - 1) * PLANE]);
                    float sh = sh2.x, sl = sl2.x;
                    ds_acc(sh, sl, sh2.y, sl2.y);
                    float yp, ye;  // wy wx
                    ds_prod(w[2 * 16 + ry[r]], w[3 * 16 + ry[r]], w[rx[r]], w[16 + rx[r]], yp, ye);
                    float pp, pe;
                    ds_prod(yp, ye, sh, sl, pp, pe);
                    ds_acc(uh, ul, pp, pe);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, uh, o);
                const float ol = __shfl_xor_sync(0xffffffffu, ul, o);
                ds_acc(uh, ul, oh, ol);
            }
            if (lane == 0)
                a.uf[3 * a.permt[p] + c] = ds_join(uh, ul) * a.scale;
        }
        __syncthreads();  // before the next component overwrites the block
    }
}

// ---- kernels: one plan, or many plans' boxes in one launch (as k_grid.cu) ----
struct GridDsBox {
    GridDsArgs a;
    const CUtensorMap *tm;  // G2P's TMA descriptor of the box's double-single grid
    int use_tma;
    int *err;
};

template <int PC>
// three blocks an SM: 80 registers (a few bytes of spill) against 124 at two
__global__ void __launch_bounds__(kP2GDsThreads, 3) k_p2g_ds(GridDsArgs a)
{
    p2g_ds_body<PC>(a, blockIdx.x);
}
template <int PC>
__global__ void __launch_bounds__(kP2GDsThreads, 3)
    k_p2g_ds_boxes(const GridDsBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    p2g_ds_body<PC>(boxes[b].a, (int)blockIdx.x - base[b]);
}
template <int PC>
__global__ void __launch_bounds__(kG2PDsThreads, 2)
    k_g2p_ds(GridDsArgs a, const __grid_constant__ CUtensorMap tmap, int use_tma, int *err)
{
    g2p_ds_body<PC>(a, blockIdx.x, &tmap, use_tma, err);
}
template <int PC>
__global__ void __launch_bounds__(kG2PDsThreads, 2)
    k_g2p_ds_boxes(const GridDsBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    const GridDsBox &x = boxes[b];
    g2p_ds_body<PC>(x.a, (int)blockIdx.x - base[b], x.tm, x.use_tma, x.err);
}

// FP64 grid -> double-single planes (all h values, then all l values)
__global__ void k_grid_split(const double *__restrict__ src, float *__restrict__ dst, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float h, l;
    ds_split(src[i], h, l);
    dst[i] = h;
    dst[n + i] = l;
}

GridDsArgs ds_args(ewald_plan_s *p)
{
    GridDsArgs a;
    a.tdat = (const dvec4 *)p->tdat;
    a.tfrc = (const float4 *)p->tfrc;
    a.wts = (const float *)p->wts;
    a.startt = p->startt;
    a.permt = p->permt;
    a.P = p->g.P;
    a.PW = ds_window_stride(p->g.P);
    a.M = p->g.M;
    a.nt = p->g.nt;
    a.KT = p->g.KT;
    a.grid = (double *)p->grid;
    a.gds = nullptr;
    a.uf = (double *)p->uf;
    a.scale = 1.0;
    return a;
}

template <int PC>
cudaError_t run_p2g_ds(const GridDsArgs &a, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (a.P != PC)
            return run_p2g_ds<PC + 1>(a, s);
        const cudaError_t e = cudaFuncSetAttribute(k_p2g_ds<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kP2GDsSmem);
        if (e != cudaSuccess)
            return e;
        k_p2g_ds<PC><<<a.nt * a.nt * a.nt, kP2GDsThreads, kP2GDsSmem, s>>>(a);
        return cudaGetLastError();
    }
}

template <int PC>
cudaError_t run_g2p_ds(const GridDsArgs &a, int *err, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (a.P != PC)
            return run_g2p_ds<PC + 1>(a, err, s);
        using G = G2PDs<PC>;
        constexpr size_t sm = G::smem;
        const cudaError_t e =
            cudaFuncSetAttribute(k_g2p_ds<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess)
            return e;
        // the double-single grid as [6][M][M][M] (h planes, then l planes);
        // one box is one component's S x RR x RR block
        CUtensorMap m;
        memset(&m, 0, sizeof(m));
        const int use_tma = grid_tensor_map(a.gds, a.M, 6, G::S, G::RR, 1, &m) ? 1 : 0;
        k_g2p_ds<PC><<<a.nt * a.nt * a.nt, kG2PDsThreads, sm, s>>>(a, m, use_tma, err);
        return cudaGetLastError();
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

bool grid_ds_supported(int P, int T, int M)
{
    return T == kT && P >= kGridDsMinP && P <= kMaxP && M <= 1024;
}

cudaError_t launch_window_ds(ewald_plan_s *p, cudaStream_t s)
{
    const int64_t n = 3 * p->N;
    if (n == 0)
        return cudaSuccess;
    k_window_ds<<<blocks_for(n, 256), 256, 0, s>>>((const dvec4 *)p->tdat, (const double *)p->wcoef_dev,
                                                  (float *)p->wts, p->N, p->g.P, p->wpoly.deg,
                                                  ds_window_stride(p->g.P));
    return cudaGetLastError();
}

cudaError_t launch_p2g_ds(ewald_plan_s *p, cudaStream_t s)
{
    return run_p2g_ds<kGridDsMinP>(ds_args(p), s);
}

cudaError_t launch_p2g_ds_with(ewald_plan_s *p, const void *tfrc, double *grid, cudaStream_t s)
{
    GridDsArgs a = ds_args(p);
    a.tfrc = (const float4 *)tfrc;
    a.grid = grid;
    return run_p2g_ds<kGridDsMinP>(a, s);
}

cudaError_t launch_g2p_ds(ewald_plan_s *p, const float *gds, double scale, cudaStream_t s)
{
    GridDsArgs a = ds_args(p);
    a.gds = gds;
    a.scale = scale;
    return run_g2p_ds<kGridDsMinP>(a, p->err, s);
}

cudaError_t launch_grid_split(const double *src, float *dst, int64_t n, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    k_grid_split<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// ---- the double-single grid stages of many plans -----------------------------
namespace {
template <typename T>
cudaError_t upload_ds(const std::vector<T> &v, T **d)
{
    *d = nullptr;
    if (v.empty())
        return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)d, sizeof(T) * v.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}
struct DsGroup {
    int kind, P;  // 0 P2G, 1 G2P
    GridDsBox *boxes = nullptr;
    int *base = nullptr, n = 0;
    unsigned grid = 0;
};
template <int PC>
cudaError_t ds_group_launch(const DsGroup &g, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (g.P != PC)
            return ds_group_launch<PC + 1>(g, s);
        if (g.kind == 0) {
            cudaError_t e = cudaFuncSetAttribute(k_p2g_ds_boxes<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kP2GDsSmem);
            if (e != cudaSuccess)
                return e;
            k_p2g_ds_boxes<PC><<<g.grid, kP2GDsThreads, kP2GDsSmem, s>>>(g.boxes, g.base, g.n);
        } else {
            constexpr size_t sm = G2PDs<PC>::smem;
            cudaError_t e = cudaFuncSetAttribute(k_g2p_ds_boxes<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess)
                return e;
            k_g2p_ds_boxes<PC><<<g.grid, kG2PDsThreads, sm, s>>>(g.boxes, g.base, g.n);
        }
        return cudaGetLastError();
    }
}
}  // namespace

struct DsGridBoxes {
    WindowJob *win = nullptr;
    int *win_base = nullptr, nwin = 0;
    unsigned win_grid = 0;
    SplitJob *split = nullptr;
    int *split_base = nullptr, nsplit = 0;
    unsigned split_grid = 0;
    std::vector<DsGroup> groups;
    CUtensorMap *maps = nullptr;
};

// The double-single plans among `plans`: grid[i] is box i's FP64 P2G output
// (its FFT input), gds[i] its double-single G2P copy.
cudaError_t ds_grid_boxes_create(ewald_plan_s *const *plans, double *const *grid, float *const *gds, int n,
                                 DsGridBoxes **out)
{
    DsGridBoxes *b = new (std::nothrow) DsGridBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    std::vector<WindowJob> win;
    std::vector<SplitJob> split;
    std::vector<int> wb(1, 0), sb(1, 0);
    std::map<std::pair<int, int>, std::vector<int>> members;
    std::vector<CUtensorMap> maps(n);
    std::vector<int> use(n, 0);
    for (int i = 0; i < n; ++i) {
        ewald_plan_s *p = plans[i];
        if (!p->grid_ds)
            continue;
        win.push_back(WindowJob{(const dvec4 *)p->tdat, (const double *)p->wcoef_dev, (float *)p->wts, p->N, p->g.P,
                                p->wpoly.deg, ds_window_stride(p->g.P)});
        wb.push_back(wb.back() + (int)blocks_for(3 * p->N, 256));
        split.push_back(SplitJob{grid[i], gds[i], 3 * p->g.nreal});
        sb.push_back(sb.back() + (int)blocks_for(3 * p->g.nreal, 256));
        members[{0, p->g.P}].push_back(i);
        members[{1, p->g.P}].push_back(i);
        memset(&maps[i], 0, sizeof(CUtensorMap));
        use[i] = grid_tensor_map(gds[i], p->g.M, 6, g2p_stride(p->g.P), kT + p->g.P - 1, 1, &maps[i]) ? 1 : 0;
    }
    b->nwin = (int)win.size();
    b->nsplit = (int)split.size();
    b->win_grid = (unsigned)wb.back();
    b->split_grid = (unsigned)sb.back();
    cudaError_t e = upload_ds(win, &b->win);
    if (e == cudaSuccess) e = upload_ds(wb, &b->win_base);
    if (e == cudaSuccess) e = upload_ds(split, &b->split);
    if (e == cudaSuccess) e = upload_ds(sb, &b->split_base);
    if (e == cudaSuccess) e = upload_ds(maps, &b->maps);
    for (auto &kv : members) {
        if (e != cudaSuccess)
            break;
        DsGroup g;
        g.kind = kv.first.first;
        g.P = kv.first.second;
        std::vector<GridDsBox> hb;
        std::vector<int> base(1, 0);
        for (int i : kv.second) {
            ewald_plan_s *p = plans[i];
            GridDsBox x;
            x.a = ds_args(p);
            x.a.grid = grid[i];
            x.a.gds = gds[i];
            x.a.scale = 1.0;
            x.tm = b->maps + i;
            x.use_tma = use[i];
            x.err = p->err;
            hb.push_back(x);
            base.push_back(base.back() + p->g.ntiles);
        }
        g.n = (int)hb.size();
        g.grid = (unsigned)base.back();
        e = upload_ds(hb, &g.boxes);
        if (e == cudaSuccess)
            e = upload_ds(base, &g.base);
        b->groups.push_back(g);
    }
    if (e != cudaSuccess) {
        ds_grid_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

// stage 0: window weights (after binning); 1: P2G; 2: the double-single copy
// of the grids (after the inverse FFT); 3: G2P
cudaError_t ds_grid_boxes_launch(const DsGridBoxes *b, int stage, cudaStream_t s)
{
    if (stage == 0 && b->nwin)
        k_window_ds_jobs<<<b->win_grid, 256, 0, s>>>(b->win, b->win_base, b->nwin);
    if (stage == 2 && b->nsplit)
        k_grid_split_jobs<<<b->split_grid, 256, 0, s>>>(b->split, b->split_base, b->nsplit);
    if (stage == 1 || stage == 3)
        for (const DsGroup &g : b->groups)
            if (g.kind == (stage == 1 ? 0 : 1)) {
                const cudaError_t e = ds_group_launch<kGridDsMinP>(g, s);
                if (e != cudaSuccess)
                    return e;
            }
    return cudaGetLastError();
}

int ds_grid_boxes_launches(const DsGridBoxes *b)
{
    return (b->nwin ? 1 : 0) + (b->nsplit ? 1 : 0) + (int)b->groups.size();
}

void ds_grid_boxes_destroy(DsGridBoxes *b)
{
    if (!b)
        return;
    void *ptrs[] = {b->win, b->win_base, b->split, b->split_base, b->maps};
    for (void *q : ptrs)
        if (q)
            cudaFree(q);
    for (DsGroup &g : b->groups) {
        if (g.boxes)
            cudaFree(g.boxes);
        if (g.base)
            cudaFree(g.base);
    }
    delete b;
}

}  // namespace ewg
