// k_grid.cu -- steps a2 (P2G, eq. (p2g)) and a6 (G2P, eq. (g2p)).
//
// Window: w(r) = w0(r1) w0(r2) w0(r3), the truncated Kaiser-Bessel w0 of
// Sec. 2.2 replaced by one degree-nu polynomial per grid bin (Sec. 4, Horner).
// A point y with anchor a (see k_bin.cu) touches grid points a + l, l < P,
// with weights w_l(delta) = w0(l + 1 - P/2 - delta), delta = frac(y/h + odd/2).
//
// P2G is written owner-computes: one block per output tile of T^3 grid points
// gathers from the points anchored in the (KT+1)^3 tiles at and before it
// (KT = ceil((P-1)/T)), so every grid value is produced once, by one block,
// in a fixed order: no atomics, no zeroing pass, bitwise-reproducible grids.
// (The paper's P2G-hybrid, Algorithm 4, is the prior art: it also keeps the
// window values in shared memory, but scatters with O(27 N) atomics.)
// The neighbour tiles' point ranges are concatenated and processed in rounds
// of 512 points: (A) two points per thread, each tested for overlap with the
// tile and compacted, (B) one thread per (point, axis) evaluates the window
// polynomial's bins, (C) threads = (two rows (y, z), (y, z + T/2) of the tile) x
// (slice of the point list) accumulate 2 x T values x 3 components in
// registers, sharing each point's x weights and force between the rows.
//
// G2P: one block per tile of anchors stages the (T+P-1)^3 grid block the
// tile's points can touch in shared memory (asynchronous copies); one warp per
// point sums its P^3 support, lanes over (y, x) pairs walking the z planes, a
// shuffle reduction at the end.
#include <cuda.h>  // CUtensorMap and its enums (types only: encoded through the runtime's driver entry point)
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "internal.h"
#include "p2g_common.h"

namespace ewg {
namespace {

struct GridArgs {
    const void *tdat, *tfrc;
    const int32_t *startt, *permt;
    const void *wcoef;
    int P, deg, M, T, nt, KT;
    void *grid;          // P2G: output grid; G2P: input grid
    void *uf;            // G2P output, user order
    double scale;        // G2P: multiplies the sum (h^3 for the bare eq. (g2p))
};

template <typename R>
__device__ __forceinline__ R horner(const R *c, int deg, R z)
{
    R p = c[deg];
    for (int k = deg - 1; k >= 0; --k)
        p = fma(p, z, c[k]);
    return p;
}

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = dvec4; };

__device__ __forceinline__ int wrapi(int i, int n) { return p2g_wrapi(i, n); }

// P2G: R = accumulation precision, G = grid element type.  PC > 0 fixes P at
// compile time: (B) then evaluates all P bins of one (point, axis) in one
// thread -- every bin shares z = 2 delta - 1, so the coefficient loads are
// warp-uniform broadcasts and the P Horner chains run side by side.
template <int T, typename R, typename G, int PC>
__device__ __forceinline__ void p2g_body(const GridArgs &a, const int tile)
{
    using R4 = typename Vec4<R>::T;
    constexpr int NT = kP2GThreads;
    constexpr int ROWS = T * T / 2;  // row pairs (y, z), (y, z + T/2)
    constexpr int SL = NT / ROWS;
    constexpr int CPT = kP2GCandidates;  // candidates per thread and round
    constexpr int B = CPT * NT;          // points per round
    constexpr int H = T / 2;
    // a warp holds one slice when ROWS is a multiple of 32: per-point tests
    // are then warp-uniform, and the tile halves [0, H), [H, T) in x and z
    // that the point's support misses are skipped as a whole
    constexpr bool kSkip = ROWS % 32 == 0;
    constexpr int PS = (PC + 3) & ~3;  // padded bins per coefficient row (PC > 0)
    extern __shared__ __align__(32) unsigned char smem[];
    R *wx = (R *)smem;              // [B][T]
    R *wy = wx + B * T;             // [B][T]
    R *wz = wy + B * T;             // [B][T]
    R *sf = wz + B * T;             // [B][4] force, padded for vector loads
    R *sd = sf + B * 4;             // [B][3] fractional offsets delta
    R *coef = sd + B * 3;           // PC = 0: [P][deg+1]; PC > 0: [deg+1][PS]
    __shared__ int soff[B];         // packed anchor offsets relative to the tile (biased)
    __shared__ int seg_start[kP2GMaxSeg], seg_pref[kP2GMaxSeg + 1];
    __shared__ int scount;

    const int nt = a.nt, P = PC > 0 ? PC : a.P, nd = a.deg + 1, KT = a.KT;
    const int side = KT + 1, nseg = side * side * side;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    if constexpr (PC > 0) {
        for (int i = threadIdx.x; i < nd * PS; i += NT) {
            const int j = i / PS, l = i - j * PS;
            coef[i] = l < PC ? ((const R *)a.wcoef)[l * nd + j] : (R)0;
        }
    } else {
        for (int i = threadIdx.x; i < P * nd; i += NT)
            coef[i] = ((const R *)a.wcoef)[i];
    }
    p2g_segment_table(a.startt, nt, KT, tx, ty, tz, seg_start, seg_pref);
    const int row = threadIdx.x % ROWS, slice = threadIdx.x / ROWS;
    const int y = row % T, z = row / T;  // rows (y, z) and (y, z + T/2)
    // FP32: the sums of x and x + 1 packed for FP32x2 FMAs, acc2[h][x / 2][c]
    constexpr bool kPack = sizeof(R) == 4 && T % 2 == 0;
    R acc[kPack ? 1 : 2][kPack ? 1 : T][3];
    float2 acc2[2][kPack ? T / 2 : 1][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if constexpr (kPack) {
#pragma unroll
            for (int x = 0; x < T / 2; ++x)
                acc2[h][x][0] = acc2[h][x][1] = acc2[h][x][2] = make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int x = 0; x < T; ++x)
                acc[h][x][0] = acc[h][x][1] = acc[h][x][2] = (R)0;
        }
    }
    __syncthreads();
    const int total = seg_pref[nseg];
    const R4 *tdat = (const R4 *)a.tdat, *tfrc = (const R4 *)a.tfrc;

    for (int base = 0; base < total; base += B) {
        if (threadIdx.x == 0)
            scount = 0;
        __syncthreads();
        // (A) CPT candidates per thread: overlap test and compaction (one
        // shared atomic per warp and candidate)
#pragma unroll
        for (int h = 0; h < CPT; ++h) {
        const int q = base + threadIdx.x + h * NT;
        bool keep = false;
        R4 td;
        int j = 0, ox = 0, oy = 0, oz = 0;
        if (q < total) {
            int dx, dy, dz;
            j = p2g_candidate(seg_start, seg_pref, nseg, KT, q, dx, dy, dz);
            td = tdat[j];
            int packed = (int)td.w;
            ox = dx * T + (packed & 15);
            oy = dy * T + ((packed >> 4) & 15);
            oz = dz * T + ((packed >> 8) & 15);
            keep = ox + P > 0 && ox < T && oy + P > 0 && oy < T && oz + P > 0 && oz < T;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        int wbase = 0;
        if ((threadIdx.x & 31) == 0 && ball)
            wbase = atomicAdd(&scount, __popc(ball));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (keep) {
            {
                int k = wbase + __popc(ball & ((1u << (threadIdx.x & 31)) - 1u));
                // offsets lie in (-P, T): bias by 32 into 6-bit fields
                soff[k] = (ox + 32) | ((oy + 32) << 6) | ((oz + 32) << 12);
                sd[k * 3] = td.x;
                sd[k * 3 + 1] = td.y;
                sd[k * 3 + 2] = td.z;
                R4 fv = tfrc[j];
                fv.w = (R)0;
                ((R4 *)sf)[k] = fv;
            }
        }
        }
        __syncthreads();
        const int n = scount;
        // (B) window values padded to the tile
        if constexpr (PC > 0) {
            // one thread per (point, axis): all P bins at once
            for (int w = threadIdx.x; w < n * 3; w += NT) {
                const int k = w / 3, d = w - 3 * k;
                const int o = ((soff[k] >> (6 * d)) & 63) - 32;
                const R zz = (R)2 * sd[k * 3 + d] - (R)1;
                R pv[PS];
                if constexpr (sizeof(R) == 4) {
                    window_bins_sym<PC, PS>(coef, nd, zz, pv);
                } else {
                    const R *cd = coef + (nd - 1) * PS;
#pragma unroll
                    for (int l = 0; l < PS; ++l)
                        pv[l] = cd[l];
                    for (int jj = nd - 2; jj >= 0; --jj) {
                        const R *cj = coef + jj * PS;
#pragma unroll
                        for (int l = 0; l < PS; ++l)
                            pv[l] = fma(pv[l], zz, cj[l]);
                    }
                }
                R *rowp = (d == 0 ? wx : (d == 1 ? wy : wz)) + k * T;
#pragma unroll
                for (int x = 0; x < T; ++x)
                    rowp[x] = (R)0;
#pragma unroll
                for (int l = 0; l < PC; ++l) {
                    const int qq = o + l;
                    if ((unsigned)qq < (unsigned)T)
                        rowp[qq] = pv[l];
                }
            }
        } else {
            // one thread per (point, axis, offset)
            for (int w = threadIdx.x; w < n * 3 * T; w += NT) {
                const int k = w / (3 * T), r = w - k * 3 * T, d = r / T, qq = r - d * T;
                const int o = ((soff[k] >> (6 * d)) & 63) - 32;
                const int l = qq - o;
                R v = (R)0;
                if (l >= 0 && l < P)
                    v = horner(coef + l * nd, a.deg, (R)2 * sd[k * 3 + d] - (R)1);
                (d == 0 ? wx : (d == 1 ? wy : wz))[k * T + qq] = v;
            }
        }
        __syncthreads();
        // (C) accumulate two rows per thread; x weights and force are shared
        for (int k = slice; k < n; k += SL) {
            bool hx0 = true, hx1 = true, hz0 = true, hz1 = true;
            if constexpr (kSkip) {
                const int so = soff[k];
                const int okx = (so & 63) - 32, okz = ((so >> 12) & 63) - 32;
                hx0 = okx < H;
                hx1 = okx + P > H;
                hz0 = okz < H;
                hz1 = okz + P > H;
            }
            const R wyk = wy[k * T + y];
            const R wz0 = wyk * wz[k * T + z], wz1 = wyk * wz[k * T + z + H];
            const R4 f = ((const R4 *)sf)[k];
            R wv[T];
#pragma unroll
            for (int x4 = 0; x4 < T / 4; ++x4) {
                const R4 qv = ((const R4 *)(wx + k * T))[x4];
                wv[4 * x4] = qv.x;
                wv[4 * x4 + 1] = qv.y;
                wv[4 * x4 + 2] = qv.z;
                wv[4 * x4 + 3] = qv.w;
            }
            if constexpr (kPack) {
                // (sum[x], sum[x + 1]) += (w[x], w[x + 1]) g: one FP32x2 FMA a pair
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 0 ? hz0 : hz1) {
                        const float wzh = h == 0 ? wz0 : wz1;
                        const float2 g[3] = {make_float2(wzh * f.x, wzh * f.x), make_float2(wzh * f.y, wzh * f.y),
                                             make_float2(wzh * f.z, wzh * f.z)};
#pragma unroll
                        for (int x = 0; x < T / 2; ++x) {
                            if (x < H / 2 ? hx0 : hx1) {
                                const float2 w2 = make_float2(wv[2 * x], wv[2 * x + 1]);
#pragma unroll
                                for (int c = 0; c < 3; ++c)
                                    acc2[h][x][c] = __ffma2_rn(w2, g[c], acc2[h][x][c]);
                            }
                        }
                    }
                }
            } else {
                if (hz0) {
                    const R g0[3] = {wz0 * f.x, wz0 * f.y, wz0 * f.z};
                    if (hx0) {
#pragma unroll
                        for (int x = 0; x < H; ++x)
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                acc[0][x][c] = fma(wv[x], g0[c], acc[0][x][c]);
                    }
                    if (hx1) {
#pragma unroll
                        for (int x = H; x < T; ++x)
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                acc[0][x][c] = fma(wv[x], g0[c], acc[0][x][c]);
                    }
                }
                if (hz1) {
                    const R g1[3] = {wz1 * f.x, wz1 * f.y, wz1 * f.z};
                    if (hx0) {
#pragma unroll
                        for (int x = 0; x < H; ++x)
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                acc[1][x][c] = fma(wv[x], g1[c], acc[1][x][c]);
                    }
                    if (hx1) {
#pragma unroll
                        for (int x = H; x < T; ++x)
#pragma unroll
                            for (int c = 0; c < 3; ++c)
                                acc[1][x][c] = fma(wv[x], g1[c], acc[1][x][c]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // reduce the slices through shared memory and store the tile
    // [SL][3][T][T][T + 1] (reuses the staging area): rows padded by one so
    // that the 32 rows (y, z) a warp writes at one x fall in 32 banks
    R *red = (R *)smem;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int x = 0; x < T; ++x)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                red[(((slice * 3 + c) * T + z + h * H) * T + y) * (T + 1) + x] =
                    kPack ? (x & 1 ? acc2[h][x / 2][c].y : acc2[h][x / 2][c].x) : acc[kPack ? 0 : h][kPack ? 0 : x][c];
    __syncthreads();
    G *grid = (G *)a.grid;
    const int64_t M = a.M, M3 = M * M * M;
    for (int o = threadIdx.x; o < 3 * T * T * T; o += NT) {
        const int x = o % T, yy = (o / T) % T, zz = (o / (T * T)) % T, c = o / (T * T * T);
        R s = 0;
#pragma unroll
        for (int qq = 0; qq < SL; ++qq)
            s += red[(((qq * 3 + c) * T + zz) * T + yy) * (T + 1) + x];
        const int64_t gx = tx * T + x, gy = ty * T + yy, gz = tz * T + zz;
        grid[c * M3 + (gz * M + gy) * M + gx] = (G)s;
    }
}

constexpr int kG2PThreads = 256;
constexpr int kMaxRounds = (kMaxP * kMaxP + 31) / 32;

// G2P: arithmetic and staging in R (the grid is given in R).  The block stages
// the (T+P-1)^3 grid block its points can touch, components interleaved per
// point, so one 16-byte (FP32) shared load returns all three.  Lanes own
// (y, x) pairs of the P x P face of a point's support and walk its P z-planes
// with one shared address each; w2[y] w1[x] is formed once per pair.
// PC > 0 fixes P at compile time (every offset into the staged block becomes
// an immediate and the loops unroll); PC = 0 reads P at run time.
template <int T, typename R, int PC>
__device__ __forceinline__ void g2p_body(const GridArgs &a, const int tile)
{
    using R4 = typename Vec4<R>::T;
    const int s0 = a.startt[tile], s1 = a.startt[tile + 1];
    if (s0 == s1)
        return;
    extern __shared__ __align__(32) unsigned char smem[];
    const int P = PC > 0 ? PC : a.P, nd = a.deg + 1, RR = T + P - 1;
    const int RR2 = RR * RR, RR3 = RR2 * RR;
    R4 *vs = (R4 *)smem;                         // [RR][RR][RR] points, (x, y, z, -)
    R *coef = (R *)(vs + RR3);                   // [P][nd]
    R *wsm = coef + P * nd;                      // per warp [3][kMaxP]
    int *tab = (int *)(wsm + (kG2PThreads / 32) * 3 * kMaxP);  // [kMaxRounds][32]
    const int nt = a.nt, M = a.M;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    for (int i = threadIdx.x; i < P * nd; i += blockDim.x)
        coef[i] = ((const R *)a.wcoef)[i];
    // (y, x) pair of lane l in round j: q = l + 32 j, packed y << 8 | x, -1 past P^2
    for (int i = threadIdx.x; i < kMaxRounds * 32; i += blockDim.x)
        tab[i] = i < P * P ? ((i / P) << 8) | (i % P) : -1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    // stage the grid block with asynchronous copies, all in flight at once:
    // warps over (component, z) planes, lanes along x; M >= P keeps one wrap
    // enough
    const R *grid = (const R *)a.grid;
    const int64_t M3 = (int64_t)M * M * M;
    int gx = tx * T + lane;  // RR = T + P - 1 <= 23 < 32
    gx -= gx >= M ? M : 0;
    for (int cz = warp; cz < 3 * RR; cz += nwarps) {
        const int c = cz / RR, z = cz - c * RR;
        int gz = tz * T + z;
        gz -= gz >= M ? M : 0;
        const R *plane = grid + c * M3 + (int64_t)gz * M * M;
        R *dst_plane = (R *)(vs + z * RR2) + c;
        if (lane < RR) {
            for (int y = 0; y < RR; ++y) {
                int gy = ty * T + y;
                gy -= gy >= M ? M : 0;
                const unsigned dst =
                    (unsigned)__cvta_generic_to_shared(dst_plane + 4 * (y * RR + lane));
                const R *src = plane + (int64_t)gy * M + gx;
                if constexpr (sizeof(R) == 4)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src));
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int nr = (P * P + 31) / 32;  // rounds of 32 (y, x) pairs
    R *w = wsm + warp * 3 * kMaxP;
    const R4 *tdat = (const R4 *)a.tdat;
    R *uf = (R *)a.uf;
    for (int p = s0 + warp; p < s1; p += nwarps) {
        R4 td = tdat[p];
        const int packed = (int)td.w;
        const int ox = packed & 15, oy = (packed >> 4) & 15, oz = (packed >> 8) & 15;
        __syncwarp();
        for (int q = lane; q < 3 * P; q += 32) {
            const int d = q / P, l = q - d * P;
            const R dl = d == 0 ? td.x : (d == 1 ? td.y : td.z);
            w[d * kMaxP + l] = horner(coef + l * nd, a.deg, (R)2 * dl - (R)1);
        }
        __syncwarp();
        R u0 = 0, u1 = 0, u2 = 0;
        if constexpr (PC > 0) {
            // z weights in registers, rows unrolled, immediate plane offsets
            R wz[PC];
#pragma unroll
            for (int k = 0; k < PC; ++k)
                wz[k] = w[2 * kMaxP + k];
            const R4 *vb = vs + (oz * RR + oy) * RR + ox;
#pragma unroll
            for (int j = 0; j < (PC * PC + 31) / 32; ++j) {
                const int q = lane + 32 * j;
                if (q < PC * PC) {
                    const int yy = q / PC, xx = q - yy * PC;
                    const R wyx = w[kMaxP + yy] * w[xx];
                    const R4 *v = vb + yy * RR + xx;
#pragma unroll
                    for (int k = 0; k < PC; ++k) {
                        const R4 qv = v[k * RR2];
                        const R ww = wyx * wz[k];
                        u0 = fma(ww, qv.x, u0);
                        u1 = fma(ww, qv.y, u1);
                        u2 = fma(ww, qv.z, u2);
                    }
                }
            }
        } else {
            for (int j = 0; j < nr; ++j) {
                const int e = tab[j * 32 + lane];
                const bool ok = e >= 0;
                const int yy = ok ? e >> 8 : 0, xx = ok ? e & 255 : 0;
                const R wyx = ok ? w[kMaxP + yy] * w[xx] : (R)0;
                const R4 *v = vs + ((oz * RR + oy + yy) * RR + ox + xx);
#pragma unroll 4
                for (int k = 0; k < P; ++k) {
                    const R4 q = v[k * RR2];
                    const R ww = wyx * w[2 * kMaxP + k];
                    u0 = fma(ww, q.x, u0);
                    u1 = fma(ww, q.y, u1);
                    u2 = fma(ww, q.z, u2);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u0 += __shfl_xor_sync(0xffffffffu, u0, o);
            u1 += __shfl_xor_sync(0xffffffffu, u1, o);
            u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        }
        if (lane == 0) {
            const int i = a.permt[p];
            const R sc = (R)a.scale;
            uf[3 * i] = u0 * sc;
            uf[3 * i + 1] = u1 * sc;
            uf[3 * i + 2] = u2 * sc;
        }
    }
}

// Planar G2P staging (FP32, T = 8).  The block stages the grid block as
// three planar arrays [c][z][y][x] with row stride S (a multiple of 4 floats,
// so 16-byte asynchronous copies fill it).  A point's P x P (y, x) pairs are
// dealt to lanes by bank: lane b takes the pairs with (S yy + xx) mod 32 = b,
// one per round, so in every round the 32 lanes read 32 different banks
// whatever the point's offset (a shift moves all banks alike).  The number of
// rounds is the largest number of pairs on one bank; S is picked to keep it
// near ceil(P^2 / 32).
constexpr int kG2PPlanarThreads = 512;  // 16 warps: two blocks fill an SM's 64 warps by half

template <int PC>
struct G2PPlanar {
    static constexpr int T = 8, RR = T + PC - 1, S = g2p_stride(PC), NR = g2p_rounds(PC, S);
    static constexpr int NCH = (RR + 3) / 4;  // 16-byte chunks per staged row
    static constexpr int PS = (PC + 3) & ~3;
    static constexpr int NW = kG2PPlanarThreads / 32;
    static constexpr size_t grid_bytes = sizeof(float) * 3 * RR * RR * S;
    __host__ __device__ static size_t smem_no_bar(int deg)
    {
        return grid_bytes + sizeof(int) * NR * 32 + sizeof(float) * (NW * 3 * PS + (deg + 1) * PS);
    }
    // plus the TMA load's mbarrier (8-byte aligned)
    __host__ __device__ static size_t bar_offset(int deg) { return (smem_no_bar(deg) + 7) & ~(size_t)7; }
    // plus 128 bytes for aligning the staged box
    __host__ __device__ static size_t smem(int deg) { return bar_offset(deg) + 8 + 128; }
};

// Bounded wait on phase 0 of an mbarrier: true once the phase completed,
// false after `limit` polls (a copy that never lands: the caller skips its
// work and raises the error flag instead of hanging the GPU).
__device__ __forceinline__ bool mbar_wait0(unsigned bar, int limit)
{
    for (int it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(bar)
                     : "memory");
        if (ok)
            return true;
    }
    return false;
}

// Shared-memory loads by 32-bit shared address, the offset an immediate.
template <int OFF>
__device__ __forceinline__ float lds_imm(unsigned addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
    return v;
}
__device__ __forceinline__ float lds_reg(unsigned addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// s_c += sum_k wz[k] v_c[z0 + k] down one staged column, two partial sums
// per component (even and odd k) for instruction-level parallelism.
template <int PLANE, int VOL, int... K>
__device__ __forceinline__ void column_sum(unsigned a, const float *wz, float (&e)[3],
                                           float (&o)[3], std::integer_sequence<int, K...>)
{
    ((K % 2 == 0
          ? (e[0] = fmaf(wz[K], lds_imm<4 * K * PLANE>(a), e[0]),
             e[1] = fmaf(wz[K], lds_imm<4 * (VOL + K * PLANE)>(a), e[1]),
             e[2] = fmaf(wz[K], lds_imm<4 * (2 * VOL + K * PLANE)>(a), e[2]))
          : (o[0] = fmaf(wz[K], lds_imm<4 * K * PLANE>(a), o[0]),
             o[1] = fmaf(wz[K], lds_imm<4 * (VOL + K * PLANE)>(a), o[1]),
             o[2] = fmaf(wz[K], lds_imm<4 * (2 * VOL + K * PLANE)>(a), o[2]))),
     ...);
}

template <int PC>
__device__ __forceinline__ void g2p_planar_body(const GridArgs &a, const int tile, const CUtensorMap *tm,
                                                int use_tma, int *err)
{
    using G = G2PPlanar<PC>;
    constexpr int T = G::T, RR = G::RR, S = G::S, NR = G::NR, NCH = G::NCH, PS = G::PS;
    constexpr int PLANE = RR * S, VOL = RR * PLANE;
    constexpr int NIT = (RR * NCH + 31) / 32;  // staging: lane iterations per plane
    const int s0 = a.startt[tile], s1 = a.startt[tile + 1];
    if (s0 == s1)
        return;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    // the staged box starts on a 128-byte boundary (the tensor copy's
    // destination alignment): the launch adds 128 bytes for the shift
    unsigned char *smem =
        smem_raw + ((128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
    float *vs = (float *)smem;                                  // [3][RR][RR][S]
    int *tab = (int *)(smem + G::grid_bytes);                   // [NR][32]
    float *wsm = (float *)(tab + NR * 32);                      // per warp [3][PS]
    float *coef = wsm + G::NW * 3 * PS;                         // [deg+1][PS]
    const unsigned vs_a = (unsigned)__cvta_generic_to_shared(vs);
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(smem + G::bar_offset(a.deg));
    const int nt = a.nt, M = a.M, nd = a.deg + 1;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Interior tiles (the block does not wrap around the periodic grid): one
    // TMA tensor copy brings the whole (c, z, y, x) box of 3 x RR x RR x S
    // floats -- the staged layout itself -- with completion on an mbarrier.
    // The others stage with 16-byte asynchronous copies that follow the wrap.
    const bool tma = use_tma && tx * T + S <= M && ty * T + RR <= M && tz * T + RR <= M;
    if (tma) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                         "r"((unsigned)G::grid_bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(vs_a),
                "l"(reinterpret_cast<uint64_t>(tm)), "r"(tx * T), "r"(ty * T), "r"(tz * T), "r"(0),
                "r"(bar_a)
                : "memory");
        }
    } else {
        // stage: one warp per (component, z) plane, lanes over (row, 16-byte
        // chunk); M a multiple of 8 keeps every chunk on one side of the periodic
        // wrap and M >= P keeps one wrap enough
        int rowoff[NIT], dstoff[NIT];
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int t = lane + 32 * it, y = t / NCH, ch = t - y * NCH;
            int gx = tx * T + 4 * ch, gy = ty * T + y;
            gx -= gx >= M ? M : 0;
            gy -= gy >= M ? M : 0;
            rowoff[it] = t < RR * NCH ? gy * M + gx : -1;
            dstoff[it] = 4 * (y * S + 4 * ch);
        }
        const float *grid = (const float *)a.grid;
        const int64_t M2 = (int64_t)M * M, M3 = M2 * M;
        for (int cz = warp; cz < 3 * RR; cz += G::NW) {
            const int c = cz / RR, z = cz - c * RR;
            int gz = tz * T + z;
            gz -= gz >= M ? M : 0;
            const float *plane = grid + c * M3 + gz * M2;
            const unsigned dplane = vs_a + 4 * cz * PLANE;
#pragma unroll
            for (int it = 0; it < NIT; ++it)
                if (rowoff[it] >= 0)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dplane + dstoff[it]),
                                 "l"(plane + rowoff[it]));
        }
        asm volatile("cp.async.commit_group;\n" ::);
    }
    // bank-dealt (y, x) pairs: lane b, round r -> the r-th row yy whose pair
    // on bank b exists, packed yy << 8 | xx, -1 past the last
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
    for (int i = threadIdx.x; i < nd * PS; i += kG2PPlanarThreads) {
        const int j = i / PS, l = i - j * PS;
        coef[i] = l < PC ? ((const float *)a.wcoef)[l * nd + j] : 0.f;
    }
    bool staged = true;
    if (tma)
        staged = mbar_wait0(bar_a, 1 << 20);
    else
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!__syncthreads_and(staged)) {  // the copy did not land: report, leave this tile's outputs
        if (threadIdx.x == 0)
            atomicOr(err, 2);
        return;
    }
    float *w = wsm + warp * 3 * PS;
    const unsigned w_a = (unsigned)__cvta_generic_to_shared(w);
    // this lane's pairs, block-invariant: column byte offset and weight addresses
    int roff[NR];
    unsigned wy_a[NR], wx_a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int e = tab[r * 32 + lane];
        const int yy = e >> 8, xx = e & 255;
        roff[r] = e >= 0 ? 4 * (yy * S + xx) : -1;
        wy_a[r] = w_a + 4 * (PS + (e >= 0 ? yy : 0));
        wx_a[r] = w_a + 4 * (e >= 0 ? xx : 0);
    }
    // window-weight lanes: (d, l) = lane and lane + 32 over 3 axes x P bins
    const int q0 = lane, q1 = lane + 32;
    const int d0 = q0 / PC, l0 = q0 - d0 * PC, d1 = q1 / PC, l1 = q1 - d1 * PC;
    const bool ok0 = q0 < 3 * PC, ok1 = q1 < 3 * PC;
    const int c0 = ok0 ? l0 : 0, c1 = ok1 ? l1 : 0;
    const float4 *tdat = (const float4 *)a.tdat;
    float *uf = (float *)a.uf;
    // each warp's next point record and output index are loaded one point
    // ahead, so their L2 latency overlaps the current point's sums
    float4 td_next = make_float4(0.f, 0.f, 0.f, 0.f);
    int i_next = 0;
    if (s0 + warp < s1) {
        td_next = tdat[s0 + warp];
        i_next = a.permt[s0 + warp];
    }
    for (int p = s0 + warp; p < s1; p += G::NW) {
        const float4 td = td_next;
        const int i = i_next;
        if (p + G::NW < s1) {
            td_next = tdat[p + G::NW];
            i_next = a.permt[p + G::NW];
        }
        const int packed = (int)td.w;
        const int ox = packed & 15, oy = (packed >> 4) & 15, oz = (packed >> 8) & 15;
        __syncwarp();
        {
            const float z0 = 2.f * (d0 == 0 ? td.x : (d0 == 1 ? td.y : td.z)) - 1.f;
            const float z1 = 2.f * (d1 == 0 ? td.x : (d1 == 1 ? td.y : td.z)) - 1.f;
            float v0 = coef[(nd - 1) * PS + c0], v1 = coef[(nd - 1) * PS + c1];
            for (int j = nd - 2; j >= 0; --j) {
                v0 = fmaf(v0, z0, coef[j * PS + c0]);
                v1 = fmaf(v1, z1, coef[j * PS + c1]);
            }
            if (ok0)
                w[d0 * PS + l0] = v0;
            if (ok1)
                w[d1 * PS + l1] = v1;
        }
        __syncwarp();
        float wz[PC];
#pragma unroll
        for (int k = 0; k < PC; ++k)
            wz[k] = w[2 * PS + k];
        const unsigned vb = vs_a + 4 * ((oz * RR + oy) * S + ox);
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (roff[r] >= 0) {
                const float wyx = lds_reg(wy_a[r]) * lds_reg(wx_a[r]);
                float e[3] = {0.f, 0.f, 0.f}, o[3] = {0.f, 0.f, 0.f};
                column_sum<PLANE, VOL>(vb + roff[r], wz, e, o, std::make_integer_sequence<int, PC>{});
                u0 = fmaf(wyx, e[0] + o[0], u0);
                u1 = fmaf(wyx, e[1] + o[1], u1);
                u2 = fmaf(wyx, e[2] + o[2], u2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u0 += __shfl_xor_sync(0xffffffffu, u0, o);
            u1 += __shfl_xor_sync(0xffffffffu, u1, o);
            u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        }
        if (lane == 0) {
            const float sc = (float)a.scale;
            uf[3 * i] = u0 * sc;
            uf[3 * i + 1] = u1 * sc;
            uf[3 * i + 2] = u2 * sc;
        }
    }
}

// FP64 G2P without staging.  An FP64 grid block of (T+P-1)^3 points x 3
// components does not fit shared memory at T = 8 from P = 13 on, and smaller
// tiles multiply the staged volume; the grid itself (3 M^3 doubles, e.g. 41 MB
// at M = 120) stays in L2, so each warp reads its point's support directly:
// lanes over the P x P (y, x) pairs (consecutive x on consecutive lanes: the
// loads of a row coalesce), z walked per lane with s_c = sum_z wz v_c, then
// u_c += wy wx s_c.  One block per tile of anchors (empty tiles exit), warps
// over the tile's points; P is a compile-time constant.
constexpr int kG2PDirectThreads = 256;

template <int T, int PC>
__device__ __forceinline__ void g2p_direct64_body(const GridArgs &a, const int tile)
{
    constexpr int NW = kG2PDirectThreads / 32, NR = (PC * PC + 31) / 32;
    const int s0 = a.startt[tile], s1 = a.startt[tile + 1];
    if (s0 == s1)
        return;
    extern __shared__ __align__(16) unsigned char smem[];
    double *coef = (double *)smem;               // [P][nd]
    double *wsm = coef + PC * (a.deg + 1);       // per warp [3][PC]
    const int nt = a.nt, M = a.M, nd = a.deg + 1;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    for (int i = threadIdx.x; i < PC * nd; i += kG2PDirectThreads)
        coef[i] = ((const double *)a.wcoef)[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *w = wsm + warp * 3 * PC;
    const double *grid = (const double *)a.grid;
    const int64_t M2 = (int64_t)M * M, M3 = M2 * M;
    const dvec4 *tdat = (const dvec4 *)a.tdat;
    double *uf = (double *)a.uf;
    for (int p = s0 + warp; p < s1; p += NW) {
        const dvec4 td = tdat[p];
        const int packed = (int)td.w;
        const int ax = tx * T + (packed & 15), ay = ty * T + ((packed >> 4) & 15),
                  az = tz * T + ((packed >> 8) & 15);
        __syncwarp();
        for (int q = lane; q < 3 * PC; q += 32) {
            const int d = q / PC, l = q - d * PC;
            const double z = 2.0 * (d == 0 ? td.x : (d == 1 ? td.y : td.z)) - 1.0;
            w[d * PC + l] = horner(coef + l * nd, a.deg, z);
        }
        __syncwarp();
        double wz[PC];
        int64_t zoff[PC];
#pragma unroll
        for (int k = 0; k < PC; ++k) {
            wz[k] = w[2 * PC + k];
            int gz = az + k;
            gz -= gz >= M ? M : 0;
            zoff[k] = gz * M2;
        }
        double u0 = 0.0, u1 = 0.0, u2 = 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int q = lane + 32 * r;
            if (q < PC * PC) {
                const int yy = q / PC, xx = q - yy * PC;
                int gy = ay + yy, gx = ax + xx;
                gy -= gy >= M ? M : 0;
                gx -= gx >= M ? M : 0;
                const double *v = grid + (int64_t)gy * M + gx;
                double s0c = 0.0, s1c = 0.0, s2c = 0.0;
#pragma unroll
                for (int k = 0; k < PC; ++k) {
                    const double *vk = v + zoff[k];
                    s0c = fma(wz[k], __ldg(vk), s0c);
                    s1c = fma(wz[k], __ldg(vk + M3), s1c);
                    s2c = fma(wz[k], __ldg(vk + 2 * M3), s2c);
                }
                const double wyx = w[PC + yy] * w[xx];
                u0 = fma(wyx, s0c, u0);
                u1 = fma(wyx, s1c, u1);
                u2 = fma(wyx, s2c, u2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u0 += __shfl_xor_sync(0xffffffffu, u0, o);
            u1 += __shfl_xor_sync(0xffffffffu, u1, o);
            u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        }
        if (lane == 0) {
            const int i = a.permt[p];
            uf[3 * i] = u0 * a.scale;
            uf[3 * i + 1] = u1 * a.scale;
            uf[3 * i + 2] = u2 * a.scale;
        }
    }
}

// ---- kernels: one plan (the tile is the block index), or many plans'
// boxes in one launch (a block finds its box by binary search over the
// boxes' block offsets and runs the same body on that box's arguments) ----
struct GridBox {
    GridArgs a;
    const CUtensorMap *tm;  // G2P's TMA descriptor of the box's grid (global memory)
    int use_tma;
    int *err;
};

template <int T, typename R, typename G, int PC>
__global__ void __launch_bounds__(kP2GThreads, sizeof(R) == 4 ? 3 : 1) k_p2g(GridArgs a)
{
    p2g_body<T, R, G, PC>(a, blockIdx.x);
}
template <int T, typename R, typename G, int PC>
__global__ void __launch_bounds__(kP2GThreads, sizeof(R) == 4 ? 3 : 1)
    k_p2g_boxes(const GridBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    p2g_body<T, R, G, PC>(boxes[b].a, (int)blockIdx.x - base[b]);
}
template <int T, typename R, int PC>
__global__ void __launch_bounds__(kG2PThreads) k_g2p(GridArgs a)
{
    g2p_body<T, R, PC>(a, blockIdx.x);
}
template <int T, typename R, int PC>
__global__ void __launch_bounds__(kG2PThreads)
    k_g2p_boxes(const GridBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    g2p_body<T, R, PC>(boxes[b].a, (int)blockIdx.x - base[b]);
}
template <int PC>
__global__ void __launch_bounds__(kG2PPlanarThreads, 2)
    k_g2p_planar(GridArgs a, const __grid_constant__ CUtensorMap tmap, int use_tma, int *err)
{
    g2p_planar_body<PC>(a, blockIdx.x, &tmap, use_tma, err);
}
template <int PC>
__global__ void __launch_bounds__(kG2PPlanarThreads, 2)
    k_g2p_planar_boxes(const GridBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    const GridBox &x = boxes[b];
    g2p_planar_body<PC>(x.a, (int)blockIdx.x - base[b], x.tm, x.use_tma, x.err);
}
template <int T, int PC>
__global__ void __launch_bounds__(kG2PDirectThreads, 2) k_g2p_direct64(GridArgs a)
{
    g2p_direct64_body<T, PC>(a, blockIdx.x);
}
template <int T, int PC>
__global__ void __launch_bounds__(kG2PDirectThreads, 2)
    k_g2p_direct64_boxes(const GridBox *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    g2p_direct64_body<T, PC>(boxes[b].a, (int)blockIdx.x - base[b]);
}

template <int T, int PC>
cudaError_t run_g2p_direct64(const GridArgs &a, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (a.P != PC)
            return run_g2p_direct64<T, PC + 1>(a, s);
        const size_t sm = sizeof(double) * ((size_t)PC * (a.deg + 1) + (kG2PDirectThreads / 32) * 3 * PC);
        k_g2p_direct64<T, PC><<<a.nt * a.nt * a.nt, kG2PDirectThreads, sm, s>>>(a);
        return cudaGetLastError();
    }
}

GridArgs grid_args(ewald_plan_s *p)
{
    GridArgs a;
    a.tdat = p->tdat;
    a.tfrc = p->tfrc;
    a.startt = p->startt;
    a.permt = p->permt;
    a.wcoef = p->wcoef_dev;
    a.P = p->g.P;
    a.deg = p->wpoly.deg;
    a.M = p->g.M;
    a.T = p->g.T;
    a.nt = p->g.nt;
    a.KT = p->g.KT;
    a.grid = p->grid;
    a.uf = p->uf;
    a.scale = 1.0;
    return a;
}

template <int T, typename R, typename G, int PC>
cudaError_t run_p2g(const GridArgs &a, cudaStream_t s)
{
    constexpr int B = kP2GThreads * kP2GCandidates;
    const size_t ncoef = PC > 0 ? (size_t)(a.deg + 1) * ((PC + 3) & ~3) : (size_t)a.P * (a.deg + 1);
    size_t stage = sizeof(R) * ((size_t)B * (3 * T + 7) + ncoef);
    size_t red = sizeof(R) * (size_t)(kP2GThreads / (T * T / 2)) * 3 * T * T * (T + 1);
    size_t sm = stage > red ? stage : red;
    cudaError_t e = cudaFuncSetAttribute(k_p2g<T, R, G, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    k_p2g<T, R, G, PC><<<a.nt * a.nt * a.nt, kP2GThreads, sm, s>>>(a);
    return cudaGetLastError();
}

// T = 8: a compile-time-P kernel for every supported P (accumulation R, grid G)
template <typename R, typename G, int PC>
cudaError_t run_p2g_fixed(const GridArgs &a, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return run_p2g<8, R, G, 0>(a, s);
    } else {
        if (a.P == PC)
            return run_p2g<8, R, G, PC>(a, s);
        return run_p2g_fixed<R, G, PC + 1>(a, s);
    }
}

template <int T, typename R, int PC>
cudaError_t run_g2p(const GridArgs &a, cudaStream_t s)
{
    using R4 = typename Vec4<R>::T;
    const int RR = T + a.P - 1;
    const size_t sm = sizeof(R4) * (size_t)RR * RR * RR +
                      sizeof(R) * ((size_t)a.P * (a.deg + 1) + (size_t)(kG2PThreads / 32) * 3 * kMaxP) +
                      sizeof(int) * kMaxRounds * 32;
    cudaError_t e =
        cudaFuncSetAttribute(k_g2p<T, R, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    k_g2p<T, R, PC><<<a.nt * a.nt * a.nt, kG2PThreads, sm, s>>>(a);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library); null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
        cudaGetLastError();
    }
    return fn;
}

}  // namespace

// TMA descriptor of a planar FP32 grid [nc][M][M][M] for G2P's staged boxes of
// (x, y, z, c) = (S, RR, RR, bc) floats: the global strides (M, M^2, M^3
// floats) and the box's inner extent (S floats) are multiples of 16 bytes, as
// the tensor copy requires.  False if the descriptor cannot be made.
bool grid_tensor_map(const void *grid, int M, int nc, int S, int RR, int bc, CUtensorMap *m)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || M % 4 != 0 || S % 4 != 0 || ((uintptr_t)grid & 15) != 0 || S > 256 || RR > 256)
        return false;
    const cuuint64_t dims[4] = {(cuuint64_t)M, (cuuint64_t)M, (cuuint64_t)M, (cuuint64_t)nc};
    const cuuint64_t strides[3] = {(cuuint64_t)M * 4, (cuuint64_t)M * M * 4, (cuuint64_t)M * M * M * 4};
    const cuuint32_t box[4] = {(cuuint32_t)S, (cuuint32_t)RR, (cuuint32_t)RR, (cuuint32_t)bc};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(grid), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

template <int PC>
cudaError_t run_g2p_planar(const GridArgs &a, int *err, cudaStream_t s)
{
    using G = G2PPlanar<PC>;
    const size_t sm = G::smem(a.deg);
    cudaError_t e =
        cudaFuncSetAttribute(k_g2p_planar<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    CUtensorMap m;
    memset(&m, 0, sizeof(m));
    const int use_tma = grid_tensor_map(a.grid, a.M, 3, G::S, G::RR, 3, &m) ? 1 : 0;
    k_g2p_planar<PC><<<a.nt * a.nt * a.nt, kG2PPlanarThreads, sm, s>>>(a, m, use_tma, err);
    return cudaGetLastError();
}

// FP32, T = 8: a compile-time-P kernel for every supported P
template <int PC>
cudaError_t run_g2p_f32_fixed(const GridArgs &a, int *err, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return run_g2p<8, float, 0>(a, s);
    } else {
        if (a.P == PC)
            return run_g2p_planar<PC>(a, err, s);
        return run_g2p_f32_fixed<PC + 1>(a, err, s);
    }
}

template <int T>
cudaError_t dispatch_p2g(ewald_plan_s *p, const GridArgs &a, cudaStream_t s)
{
    if constexpr (T == 8) {
        // FP64: the run-time-P kernel (the compile-time one spills, measured slower)
        if (p->near64)
            return run_p2g<8, double, double, 0>(a, s);
        if (p->fft64)
            return run_p2g_fixed<float, double, 2>(a, s);
        return run_p2g_fixed<float, float, 2>(a, s);
    } else {
        if (p->near64)
            return run_p2g<T, double, double, 0>(a, s);
        if (p->fft64)
            return run_p2g<T, float, double, 0>(a, s);
        return run_p2g<T, float, float, 0>(a, s);
    }
}

}  // namespace

cudaError_t launch_p2g(ewald_plan_s *p, cudaStream_t s)
{
    if (p->grid_ds)
        return launch_p2g_ds(p, s);
    GridArgs a = grid_args(p);
    return p->g.T == 8 ? dispatch_p2g<8>(p, a, s) : dispatch_p2g<4>(p, a, s);
}

cudaError_t launch_p2g_with(ewald_plan_s *p, const void *tfrc, void *grid, cudaStream_t s)
{
    if (p->grid_ds)
        return cudaErrorNotSupported;
    GridArgs a = grid_args(p);
    a.tfrc = tfrc;
    a.grid = grid;
    return p->g.T == 8 ? dispatch_p2g<8>(p, a, s) : dispatch_p2g<4>(p, a, s);
}

// G2P from a grid in the kernels' precision (FP64 when near64, else FP32;
// double-single h and l planes for the double-single kernels).
cudaError_t launch_g2p(ewald_plan_s *p, const void *grid, double scale, cudaStream_t s)
{
    if (p->grid_ds)
        return launch_g2p_ds(p, (const float *)grid, scale, s);
    GridArgs a = grid_args(p);
    a.grid = const_cast<void *>(grid);
    a.scale = scale;
    if (p->near64)
        return p->g.T == 8 ? run_g2p_direct64<8, 2>(a, s) : run_g2p_direct64<4, 2>(a, s);
    return p->g.T == 8 ? run_g2p_f32_fixed<2>(a, p->err, s) : run_g2p<4, float, 0>(a, s);
}

// ---- the grid stages of many plans, one launch per kernel variant -------
namespace {

// one launch: boxes of one kernel instantiation
struct GridGroup {
    int kind;       // 0 P2G, 1 G2P
    int fft64;      // the boxes' FFT precision (launches are issued per FFT precision)
    int prec;       // P2G: 0 (FP32, FP32 grid), 1 (FP32, FP64 grid), 2 (FP64); G2P: 0 FP32, 2 FP64
    int T, P, deg;  // tile, support, largest window degree of the group's boxes
    GridBox *boxes = nullptr;
    int *base = nullptr;
    int n = 0;
    unsigned grid = 0;
};

template <int T, typename R, int PC>
size_t p2g_smem(int P, int deg)
{
    constexpr int B = kP2GThreads * kP2GCandidates;
    const size_t ncoef = PC > 0 ? (size_t)(deg + 1) * ((PC + 3) & ~3) : (size_t)P * (deg + 1);
    const size_t stage = sizeof(R) * ((size_t)B * (3 * T + 7) + ncoef);
    const size_t red = sizeof(R) * (size_t)(kP2GThreads / (T * T / 2)) * 3 * T * T * (T + 1);
    return stage > red ? stage : red;
}

template <int T, typename R, typename G, int PC>
cudaError_t p2g_group(const GridGroup &g, cudaStream_t s)
{
    const size_t sm = p2g_smem<T, R, PC>(g.P, g.deg);
    cudaError_t e = cudaFuncSetAttribute(k_p2g_boxes<T, R, G, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    k_p2g_boxes<T, R, G, PC><<<g.grid, kP2GThreads, sm, s>>>(g.boxes, g.base, g.n);
    return cudaGetLastError();
}
template <typename R, typename G, int PC>
cudaError_t p2g_group_fixed(const GridGroup &g, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return p2g_group<8, R, G, 0>(g, s);
    } else {
        if (g.P == PC)
            return p2g_group<8, R, G, PC>(g, s);
        return p2g_group_fixed<R, G, PC + 1>(g, s);
    }
}
template <int T, typename R, int PC>
cudaError_t g2p_group_generic(const GridGroup &g, cudaStream_t s)
{
    using R4 = typename Vec4<R>::T;
    const int RR = T + g.P - 1;
    const size_t sm = sizeof(R4) * (size_t)RR * RR * RR +
                      sizeof(R) * ((size_t)g.P * (g.deg + 1) + (size_t)(kG2PThreads / 32) * 3 * kMaxP) +
                      sizeof(int) * kMaxRounds * 32;
    cudaError_t e = cudaFuncSetAttribute(k_g2p_boxes<T, R, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    k_g2p_boxes<T, R, PC><<<g.grid, kG2PThreads, sm, s>>>(g.boxes, g.base, g.n);
    return cudaGetLastError();
}
template <int PC>
cudaError_t g2p_group_planar(const GridGroup &g, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return g2p_group_generic<8, float, 0>(g, s);
    } else {
        if (g.P != PC)
            return g2p_group_planar<PC + 1>(g, s);
        const size_t sm = G2PPlanar<PC>::smem(g.deg);
        cudaError_t e = cudaFuncSetAttribute(k_g2p_planar_boxes<PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess)
            return e;
        k_g2p_planar_boxes<PC><<<g.grid, kG2PPlanarThreads, sm, s>>>(g.boxes, g.base, g.n);
        return cudaGetLastError();
    }
}
template <int T, int PC>
cudaError_t g2p_group_direct64(const GridGroup &g, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (g.P != PC)
            return g2p_group_direct64<T, PC + 1>(g, s);
        const size_t sm = sizeof(double) * ((size_t)PC * (g.deg + 1) + (kG2PDirectThreads / 32) * 3 * PC);
        k_g2p_direct64_boxes<T, PC><<<g.grid, kG2PDirectThreads, sm, s>>>(g.boxes, g.base, g.n);
        return cudaGetLastError();
    }
}

cudaError_t launch_group(const GridGroup &g, cudaStream_t s)
{
    if (g.kind == 0) {  // P2G
        if (g.T == 8) {
            if (g.prec == 2)
                return p2g_group<8, double, double, 0>(g, s);
            return g.prec == 1 ? p2g_group_fixed<float, double, 2>(g, s) : p2g_group_fixed<float, float, 2>(g, s);
        }
        if (g.prec == 2)
            return p2g_group<4, double, double, 0>(g, s);
        return g.prec == 1 ? p2g_group<4, float, double, 0>(g, s) : p2g_group<4, float, float, 0>(g, s);
    }
    if (g.prec == 2)  // FP64 G2P from the grid in L2
        return g.T == 8 ? g2p_group_direct64<8, 2>(g, s) : g2p_group_direct64<4, 2>(g, s);
    return g.T == 8 ? g2p_group_planar<2>(g, s) : g2p_group_generic<4, float, 0>(g, s);
}

}  // namespace

struct GridBoxes {
    std::vector<GridGroup> groups;  // P2G groups first, then G2P groups
    int np2g = 0;
    CUtensorMap *maps = nullptr;    // G2P TMA descriptors, one per box (device)
};

// grid[i]: box i's P2G output (FP32 or FP64 as its plan's FFT); g2p[i]: its
// G2P input (FP32 for FP32 kernels, FP64 for FP64 ones).  Plans with
// double-single grid kernels are left to ds_grid_boxes_create.
cudaError_t grid_boxes_create(ewald_plan_s *const *plans, void *const *grid, void *const *g2p, int n, GridBoxes **out)
{
    GridBoxes *b = new (std::nothrow) GridBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    struct Key {
        int kind, prec, T, P, fft64;
        bool operator<(const Key &o) const
        {
            return std::make_pair(std::make_pair(std::make_pair(kind, prec), std::make_pair(T, P)), fft64) <
                   std::make_pair(std::make_pair(std::make_pair(o.kind, o.prec), std::make_pair(o.T, o.P)), o.fft64);
        }
    };
    std::map<Key, std::vector<int>> members;
    std::vector<CUtensorMap> maps(n);
    std::vector<int> use(n, 0);
    for (int i = 0; i < n; ++i) {
        ewald_plan_s *p = plans[i];
        if (p->grid_ds)
            continue;
        const int prec = p->near64 ? 2 : (p->fft64 ? 1 : 0), f64 = p->fft64 ? 1 : 0;
        members[Key{0, prec, p->g.T, p->g.P, f64}].push_back(i);
        members[Key{1, p->near64 ? 2 : 0, p->g.T, p->g.P, f64}].push_back(i);
        memset(&maps[i], 0, sizeof(CUtensorMap));
        if (!p->near64 && p->g.T == 8 && p->g.P <= kMaxP)
            use[i] = grid_tensor_map(g2p[i], p->g.M, 3, g2p_stride(p->g.P), 8 + p->g.P - 1, 3, &maps[i]) ? 1 : 0;
    }
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMalloc(&b->maps, sizeof(CUtensorMap) * n);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->maps, maps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice);
    }
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass)
        for (auto &kv : members) {
            if (kv.first.kind != pass)
                continue;
            GridGroup g;
            g.kind = kv.first.kind;
            g.prec = kv.first.prec;
            g.T = kv.first.T;
            g.P = kv.first.P;
            g.fft64 = kv.first.fft64;
            g.deg = 0;
            std::vector<GridBox> hb;
            std::vector<int> base(1, 0);
            for (int i : kv.second) {
                ewald_plan_s *p = plans[i];
                GridBox x;
                x.a = grid_args(p);
                x.a.grid = pass == 0 ? grid[i] : g2p[i];
                x.a.scale = 1.0;
                x.tm = b->maps + i;
                x.use_tma = use[i];
                x.err = p->err;
                hb.push_back(x);
                base.push_back(base.back() + p->g.ntiles);
                g.deg = std::max(g.deg, p->wpoly.deg);
            }
            g.n = (int)hb.size();
            g.grid = (unsigned)base.back();
            e = cudaMalloc(&g.boxes, sizeof(GridBox) * hb.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(g.boxes, hb.data(), sizeof(GridBox) * hb.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMalloc(&g.base, sizeof(int) * base.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(g.base, base.data(), sizeof(int) * base.size(), cudaMemcpyHostToDevice);
            b->groups.push_back(g);
            if (pass == 0)
                b->np2g++;
        }
    if (e != cudaSuccess) {
        grid_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t grid_boxes_launch(const GridBoxes *b, int kind, cudaStream_t s, int fft64)
{
    for (const GridGroup &g : b->groups)
        if (g.kind == kind && g.fft64 == fft64) {
            const cudaError_t e = launch_group(g, s);
            if (e != cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

int grid_boxes_launches(const GridBoxes *b) { return (int)b->groups.size(); }

void grid_boxes_destroy(GridBoxes *b)
{
    if (!b)
        return;
    for (GridGroup &g : b->groups) {
        if (g.boxes)
            cudaFree(g.boxes);
        if (g.base)
            cudaFree(g.base);
    }
    if (b->maps)
        cudaFree(b->maps);
    delete b;
}

}  // namespace ewg
