// k_p2g9.cu -- step a2 (P2G, eq. (p2g)) of the combined single and double
// layer (Sec. 2.3) in one pass: the Stokeslet forces f and the double layer's
// two density triples spread onto their three 3-component grids together, so
// every point's window rows are evaluated once per output tile instead of
// once per triple.
//
// Same owner-computes scheme as the 3-component P2G (k_grid.cu): one block of
// 256 threads per 8^3 output tile gathers, in rounds of 512 candidates, from
// the points anchored in the (KT+1)^3 tiles at and before it: (A) overlap test
// and compaction, (B) one thread per (point, axis) evaluates its P window bins
// (compile-time P, FP32x2 Horner), (C) a thread owns one row (y, z) of the
// tile and its 8 x 9 sums (FP32x2 pairs over x), reading each point's x
// weights and nine densities once.  A warp's 32 rows share one z half, so a
// point whose support misses that half is skipped by the whole warp.  The
// slices' partial sums are reduced in shared memory in a fixed order: each
// grid value is written once, bitwise reproducibly.  FP32 accumulation; the
// grids are FP32 or FP64 (G).
#include <stdint.h>

#include "internal.h"
#include "p2g_common.h"

namespace ewg {
namespace {

constexpr int kT9 = 8;                     // tile edge
constexpr int kRows9 = kT9 * kT9;          // rows (y, z) of a tile
constexpr int kSl9 = kP2GThreads / kRows9;  // slices of the point list
constexpr int kB9 = kP2GThreads * kP2GCandidates;
constexpr int kNc9 = 9;                    // three triples

struct P2G9Args {
    const float4 *tdat;       // per point: delta (x, y, z) and packed anchor offsets (w)
    const float4 *frc[3];     // per point and triple: the three values (w unused)
    const int32_t *startt;    // tile start offsets (nt^3 + 1)
    const float *wcoef;       // window polynomial, [P][deg + 1]
    void *grid[3];            // three 3-component grids, component-major M^3 each
    int deg, M, nt, KT;
};

template <typename G, int PC>
__global__ void __launch_bounds__(kP2GThreads, 2) k_p2g9(P2G9Args a)
{
    constexpr int T = kT9, NT = kP2GThreads, B = kB9, H = T / 2, PS = (PC + 3) & ~3;
    extern __shared__ __align__(32) unsigned char smem[];
    float *wx = (float *)smem;   // [B][T]
    float *wy = wx + B * T;      // [B][T]
    float *wz = wy + B * T;      // [B][T]
    float4 *sf = (float4 *)(wz + B * T);  // [B][3]
    float *sd = (float *)(sf + B * 3);    // [B][3] fractional offsets delta
    float *coef = sd + B * 3;             // [deg+1][PS]
    __shared__ int soff[B];
    __shared__ int seg_start[kP2GMaxSeg], seg_pref[kP2GMaxSeg + 1];
    __shared__ int scount;

    const int tile = blockIdx.x, nt = a.nt, nd = a.deg + 1, KT = a.KT;
    const int side = KT + 1, nseg = side * side * side;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    for (int i = threadIdx.x; i < nd * PS; i += NT) {
        const int j = i / PS, l = i - j * PS;
        coef[i] = l < PC ? a.wcoef[l * nd + j] : 0.f;
    }
    p2g_segment_table(a.startt, nt, KT, tx, ty, tz, seg_start, seg_pref);
    const int row = threadIdx.x % kRows9, slice = threadIdx.x / kRows9;
    const int y = row % T, z = row / T;
    const bool zhi = z >= H;  // the same for the 32 rows of a warp
    float2 acc[T / 2][kNc9];
#pragma unroll
    for (int x = 0; x < T / 2; ++x)
#pragma unroll
        for (int c = 0; c < kNc9; ++c)
            acc[x][c] = make_float2(0.f, 0.f);
    __syncthreads();
    const int total = seg_pref[nseg];

    for (int base = 0; base < total; base += B) {
        if (threadIdx.x == 0)
            scount = 0;
        __syncthreads();
        // (A) overlap test and compaction
#pragma unroll
        for (int h = 0; h < kP2GCandidates; ++h) {
            const int q = base + threadIdx.x + h * NT;
            bool keep = false;
            float4 td = make_float4(0.f, 0.f, 0.f, 0.f);
            int j = 0, ox = 0, oy = 0, oz = 0;
            if (q < total) {
                int dx, dy, dz;
                j = p2g_candidate(seg_start, seg_pref, nseg, KT, q, dx, dy, dz);
                td = a.tdat[j];
                const int packed = (int)td.w;
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
                soff[k] = (ox + 32) | ((oy + 32) << 6) | ((oz + 32) << 12);
                sd[k * 3] = td.x;
                sd[k * 3 + 1] = td.y;
                sd[k * 3 + 2] = td.z;
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    sf[k * 3 + t] = a.frc[t][j];
            }
        }
        __syncthreads();
        const int n = scount;
        // (B) window rows padded to the tile: one thread per (point, axis)
        for (int w = threadIdx.x; w < n * 3; w += NT) {
            const int k = w / 3, d = w - 3 * k;
            const int o = ((soff[k] >> (6 * d)) & 63) - 32;
            const float zz = 2.f * sd[k * 3 + d] - 1.f;
            float pv[PS];
            window_bins_sym<PC, PS>(coef, nd, zz, pv);
            float *rowp = (d == 0 ? wx : (d == 1 ? wy : wz)) + k * T;
#pragma unroll
            for (int x = 0; x < T; ++x)
                rowp[x] = 0.f;
#pragma unroll
            for (int l = 0; l < PC; ++l) {
                const int qq = o + l;
                if ((unsigned)qq < (unsigned)T)
                    rowp[qq] = pv[l];
            }
        }
        __syncthreads();
        // (C) one row (y, z) per thread, nine sums per x
        for (int k = slice; k < n; k += kSl9) {
            const int so = soff[k];
            const int okx = (so & 63) - 32, okz = ((so >> 12) & 63) - 32;
            const bool hz = zhi ? okz + PC > H : okz < H;
            if (!hz)
                continue;  // warp-uniform
            const bool hx0 = okx < H, hx1 = okx + PC > H;
            const float wyz = wy[k * T + y] * wz[k * T + z];
            float g[kNc9];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const float4 fv = sf[k * 3 + t];
                g[3 * t] = wyz * fv.x;
                g[3 * t + 1] = wyz * fv.y;
                g[3 * t + 2] = wyz * fv.z;
            }
            const float4 qa = ((const float4 *)(wx + k * T))[0], qb = ((const float4 *)(wx + k * T))[1];
            const float2 w2[T / 2] = {make_float2(qa.x, qa.y), make_float2(qa.z, qa.w), make_float2(qb.x, qb.y),
                                      make_float2(qb.z, qb.w)};
#pragma unroll
            for (int x = 0; x < T / 2; ++x) {
                if (x < H / 2 ? hx0 : hx1) {
#pragma unroll
                    for (int c = 0; c < kNc9; ++c)
                        acc[x][c] = __ffma2_rn(w2[x], make_float2(g[c], g[c]), acc[x][c]);
                }
            }
        }
        __syncthreads();
    }
    // reduce the slices through shared memory (reusing the staging area) and
    // store the three tiles
    float *red = (float *)smem;  // [kSl9][kNc9][T][T][T + 1]: rows padded by one (bank-conflict-free writes)
#pragma unroll
    for (int x = 0; x < T; ++x)
#pragma unroll
        for (int c = 0; c < kNc9; ++c)
            red[(((slice * kNc9 + c) * T + z) * T + y) * (T + 1) + x] = (x & 1) ? acc[x / 2][c].y : acc[x / 2][c].x;
    __syncthreads();
    const int64_t M = a.M, M3 = M * M * M;
    for (int o = threadIdx.x; o < kNc9 * T * T * T; o += NT) {
        const int x = o % T, yy = (o / T) % T, zz = (o / (T * T)) % T, c = o / (T * T * T);
        float s = 0.f;
#pragma unroll
        for (int qq = 0; qq < kSl9; ++qq)
            s += red[(((qq * kNc9 + c) * T + zz) * T + yy) * (T + 1) + x];
        const int64_t gx = tx * T + x, gy = ty * T + yy, gz = tz * T + zz;
        const int t = c / 3, cc = c - 3 * t;
        G *gp = (G *)(t == 0 ? a.grid[0] : (t == 1 ? a.grid[1] : a.grid[2]));  // no dynamic parameter index
        gp[cc * M3 + (gz * M + gy) * M + gx] = (G)s;
    }
}

size_t p2g9_smem(int PS, int deg)
{
    const size_t stage = sizeof(float) * ((size_t)kB9 * (3 * kT9 + 12 + 3) + (size_t)(deg + 1) * PS);
    const size_t red = sizeof(float) * (size_t)kSl9 * kNc9 * kT9 * kT9 * (kT9 + 1);
    return stage > red ? stage : red;
}

template <typename G, int PC>
cudaError_t run_p2g9(const P2G9Args &a, int P, cudaStream_t s)
{
    if constexpr (PC > kMaxP) {
        return cudaErrorInvalidValue;
    } else {
        if (P != PC)
            return run_p2g9<G, PC + 1>(a, P, s);
        const size_t sm = p2g9_smem((PC + 3) & ~3, a.deg);
        cudaError_t e = cudaFuncSetAttribute(k_p2g9<G, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess)
            return e;
        k_p2g9<G, PC><<<a.nt * a.nt * a.nt, kP2GThreads, sm, s>>>(a);
        return cudaGetLastError();
    }
}

}  // namespace

bool p2g9_supported(const ewald_plan_s *p)
{
    return !p->near64 && !p->grid_ds && p->g.T == kT9 && p->g.P >= 2 && p->g.P <= kMaxP;
}

cudaError_t launch_p2g9(ewald_plan_s *p, const void *dl_tf, void *dl_grid, cudaStream_t s)
{
    if (!p2g9_supported(p))
        return cudaErrorNotSupported;
    P2G9Args a;
    a.tdat = (const float4 *)p->tdat;
    a.frc[0] = (const float4 *)p->tfrc;
    a.frc[1] = (const float4 *)dl_tf;
    a.frc[2] = (const float4 *)dl_tf + p->N;
    a.startt = p->startt;
    a.wcoef = (const float *)p->wcoef_dev;
    const size_t gs = p->fft64 ? sizeof(double) : sizeof(float);
    a.grid[0] = p->grid;
    a.grid[1] = dl_grid;
    a.grid[2] = (char *)dl_grid + 3 * gs * (size_t)p->g.nreal;
    a.deg = p->wpoly.deg;
    a.M = p->g.M;
    a.nt = p->g.nt;
    a.KT = p->g.KT;
    return p->fft64 ? run_p2g9<double, 2>(a, p->g.P, s) : run_p2g9<float, 2>(a, p->g.P, s);
}

}  // namespace ewg
