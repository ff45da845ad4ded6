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
// Threads are (row = (y, z) of the tile) x (slice of the point list); each
// keeps its row of T values x 3 components in registers.
//
// G2P: one block per tile of anchors stages the (T+P-1)^3 grid block the
// tile's points can touch in shared memory; one warp per point sums its P^3
// support (lanes over (z, y) rows, a shuffle reduction at the end).
#include <math.h>

#include "internal.h"

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
        p = p * z + c[k];
    return p;
}

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = dvec4; };

constexpr int kP2GThreads = 256;

// P2G: R = accumulation precision, G = grid element type.
template <int T, typename R, typename G>
__global__ void __launch_bounds__(kP2GThreads) k_p2g(GridArgs a)
{
    using R4 = typename Vec4<R>::T;
    constexpr int ROWS = T * T;
    constexpr int SL = kP2GThreads / ROWS;
    constexpr int B = kP2GThreads;  // points staged per round
    extern __shared__ __align__(32) unsigned char smem[];
    R *wx = (R *)smem;              // [B][T]
    R *wy = wx + B * T;             // [B][T]
    R *wz = wy + B * T;             // [B][T]
    R *sf = wz + B * T;             // [B][3]
    R *coef = sf + B * 3;           // [P][deg+1]
    __shared__ int scount;

    const int nt = a.nt, P = a.P, nd = a.deg + 1;
    const int tile = blockIdx.x;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    for (int i = threadIdx.x; i < P * nd; i += blockDim.x)
        coef[i] = ((const R *)a.wcoef)[i];
    const int row = threadIdx.x % ROWS, slice = threadIdx.x / ROWS;
    const int y = row % T, z = row / T;
    R acc[T][3];
#pragma unroll
    for (int x = 0; x < T; ++x)
        acc[x][0] = acc[x][1] = acc[x][2] = (R)0;

    const R4 *tdat = (const R4 *)a.tdat, *tfrc = (const R4 *)a.tfrc;
    for (int dz = -a.KT; dz <= 0; ++dz)
        for (int dy = -a.KT; dy <= 0; ++dy)
            for (int dx = -a.KT; dx <= 0; ++dx) {
                int nx = (tx + dx) % nt, ny = (ty + dy) % nt, nz = (tz + dz) % nt;
                nx += nx < 0 ? nt : 0;
                ny += ny < 0 ? nt : 0;
                nz += nz < 0 ? nt : 0;
                int nb = (nz * nt + ny) * nt + nx;
                int s0 = a.startt[nb], s1 = a.startt[nb + 1];
                for (int base = s0; base < s1; base += B) {
                    __syncthreads();
                    if (threadIdx.x == 0)
                        scount = 0;
                    __syncthreads();
                    int j = base + threadIdx.x;
                    if (j < s1) {
                        R4 td = tdat[j];
                        int packed = (int)td.w;
                        // anchor offsets relative to this output tile's origin
                        int ox = dx * T + (packed & 15);
                        int oy = dy * T + ((packed >> 4) & 15);
                        int oz = dz * T + ((packed >> 8) & 15);
                        if (ox + P > 0 && ox < T && oy + P > 0 && oy < T && oz + P > 0 && oz < T) {
                            int k = atomicAdd(&scount, 1);
                            R zx = (R)2 * td.x - (R)1, zy = (R)2 * td.y - (R)1, zz = (R)2 * td.z - (R)1;
#pragma unroll
                            for (int q = 0; q < T; ++q) {
                                int lx = q - ox, ly = q - oy, lz = q - oz;
                                wx[k * T + q] = (lx >= 0 && lx < P) ? horner(coef + lx * nd, a.deg, zx) : (R)0;
                                wy[k * T + q] = (ly >= 0 && ly < P) ? horner(coef + ly * nd, a.deg, zy) : (R)0;
                                wz[k * T + q] = (lz >= 0 && lz < P) ? horner(coef + lz * nd, a.deg, zz) : (R)0;
                            }
                            R4 fv = tfrc[j];
                            sf[k * 3] = fv.x;
                            sf[k * 3 + 1] = fv.y;
                            sf[k * 3 + 2] = fv.z;
                        }
                    }
                    __syncthreads();
                    const int n = scount;
                    for (int k = slice; k < n; k += SL) {
                        R wyz = wy[k * T + y] * wz[k * T + z];
                        if (wyz != (R)0) {
                            R f0 = wyz * sf[k * 3], f1 = wyz * sf[k * 3 + 1], f2 = wyz * sf[k * 3 + 2];
#pragma unroll
                            for (int x = 0; x < T; ++x) {
                                R w = wx[k * T + x];
                                acc[x][0] += w * f0;
                                acc[x][1] += w * f1;
                                acc[x][2] += w * f2;
                            }
                        }
                    }
                }
            }
    // reduce the slices through shared memory and store the tile
    __syncthreads();
    R *red = (R *)smem;  // [SL][3][T][T][T]  (reuses the staging area)
#pragma unroll
    for (int x = 0; x < T; ++x)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            red[((slice * 3 + c) * T + z) * T * T + y * T + x] = acc[x][c];
    __syncthreads();
    G *grid = (G *)a.grid;
    const int64_t M = a.M, M3 = M * M * M;
    for (int o = threadIdx.x; o < 3 * T * T * T; o += blockDim.x) {
        int x = o % T, yy = (o / T) % T, zz = (o / (T * T)) % T, c = o / (T * T * T);
        R s = 0;
        for (int q = 0; q < SL; ++q)
            s += red[((q * 3 + c) * T + zz) * T * T + yy * T + x];
        int64_t gx = tx * T + x, gy = ty * T + yy, gz = tz * T + zz;
        grid[c * M3 + (gz * M + gy) * M + gx] = (G)s;
    }
}

constexpr int kG2PThreads = 128;

// G2P: R = arithmetic precision, G = grid element type.
template <int T, typename R, typename G>
__global__ void __launch_bounds__(kG2PThreads) k_g2p(GridArgs a)
{
    using R4 = typename Vec4<R>::T;
    const int tile = blockIdx.x;
    const int s0 = a.startt[tile], s1 = a.startt[tile + 1];
    if (s0 == s1)
        return;
    extern __shared__ __align__(32) unsigned char smem[];
    const int P = a.P, nd = a.deg + 1, RR = T + P - 1;
    const int RR3 = RR * RR * RR;
    R *vs = (R *)smem;                 // [3][RR][RR][RR]
    R *coef = vs + 3 * RR3;            // [P][nd]
    R *wsm = coef + P * nd;            // per warp [3][kMaxP]
    const int nt = a.nt;
    const int tx = tile % nt, ty = (tile / nt) % nt, tz = tile / (nt * nt);
    for (int i = threadIdx.x; i < P * nd; i += blockDim.x)
        coef[i] = ((const R *)a.wcoef)[i];
    const G *grid = (const G *)a.grid;
    const int64_t M = a.M, M3 = M * M * M;
    for (int i = threadIdx.x; i < 3 * RR3; i += blockDim.x) {
        int x = i % RR, y = (i / RR) % RR, z = (i / (RR * RR)) % RR, c = i / RR3;
        int64_t gx = (tx * T + x) % M, gy = (ty * T + y) % M, gz = (tz * T + z) % M;
        vs[i] = (R)grid[c * M3 + (gz * M + gy) * M + gx];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    R *w = wsm + warp * 3 * kMaxP;
    const R4 *tdat = (const R4 *)a.tdat;
    R *uf = (R *)a.uf;
    for (int p = s0 + warp; p < s1; p += nwarps) {
        R4 td = tdat[p];
        int packed = (int)td.w;
        int ox = packed & 15, oy = (packed >> 4) & 15, oz = (packed >> 8) & 15;
        __syncwarp();
        for (int q = lane; q < 3 * P; q += 32) {
            int d = q / P, l = q % P;
            R dl = d == 0 ? td.x : (d == 1 ? td.y : td.z);
            w[d * kMaxP + l] = horner(coef + l * nd, a.deg, (R)2 * dl - (R)1);
        }
        __syncwarp();
        R u0 = 0, u1 = 0, u2 = 0;
        for (int q = lane; q < P * P; q += 32) {
            int k = q / P, l = q % P;  // k: z offset, l: y offset
            R wkl = w[2 * kMaxP + k] * w[kMaxP + l];
            int base = ((oz + k) * RR + (oy + l)) * RR + ox;
            R s0r = 0, s1r = 0, s2r = 0;
            for (int m = 0; m < P; ++m) {
                R wm = w[m];
                s0r += wm * vs[base + m];
                s1r += wm * vs[RR3 + base + m];
                s2r += wm * vs[2 * RR3 + base + m];
            }
            u0 += wkl * s0r;
            u1 += wkl * s1r;
            u2 += wkl * s2r;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u0 += __shfl_xor_sync(0xffffffffu, u0, o);
            u1 += __shfl_xor_sync(0xffffffffu, u1, o);
            u2 += __shfl_xor_sync(0xffffffffu, u2, o);
        }
        if (lane == 0) {
            int i = a.permt[p];
            R sc = (R)a.scale;
            uf[3 * i] = u0 * sc;
            uf[3 * i + 1] = u1 * sc;
            uf[3 * i + 2] = u2 * sc;
        }
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

template <int T, typename R, typename G>
cudaError_t run_p2g(const GridArgs &a, cudaStream_t s)
{
    constexpr int B = kP2GThreads;
    size_t stage = sizeof(R) * ((size_t)B * (3 * T + 3) + (size_t)a.P * (a.deg + 1));
    size_t red = sizeof(R) * (size_t)(kP2GThreads / (T * T)) * 3 * T * T * T;
    size_t sm = stage > red ? stage : red;
    cudaError_t e = cudaFuncSetAttribute(k_p2g<T, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess)
        return e;
    k_p2g<T, R, G><<<a.nt * a.nt * a.nt, kP2GThreads, sm, s>>>(a);
    return cudaGetLastError();
}

template <int T, typename R, typename G>
cudaError_t run_g2p(const GridArgs &a, cudaStream_t s)
{
    int RR = T + a.P - 1;
    size_t sm = sizeof(R) * ((size_t)3 * RR * RR * RR + (size_t)a.P * (a.deg + 1) +
                             (size_t)(kG2PThreads / 32) * 3 * kMaxP);
    cudaError_t e = cudaFuncSetAttribute(k_g2p<T, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess)
        return e;
    k_g2p<T, R, G><<<a.nt * a.nt * a.nt, kG2PThreads, sm, s>>>(a);
    return cudaGetLastError();
}

template <int T>
cudaError_t dispatch_p2g(ewald_plan_s *p, const GridArgs &a, cudaStream_t s)
{
    if (p->near64)
        return run_p2g<T, double, double>(a, s);
    if (p->fft64)
        return run_p2g<T, float, double>(a, s);
    return run_p2g<T, float, float>(a, s);
}

template <int T>
cudaError_t dispatch_g2p(ewald_plan_s *p, const GridArgs &a, bool grid64, cudaStream_t s)
{
    if (p->near64)
        return grid64 ? run_g2p<T, double, double>(a, s) : run_g2p<T, double, float>(a, s);
    return grid64 ? run_g2p<T, float, double>(a, s) : run_g2p<T, float, float>(a, s);
}

}  // namespace

cudaError_t launch_p2g(ewald_plan_s *p, cudaStream_t s)
{
    GridArgs a = grid_args(p);
    return p->g.T == 8 ? dispatch_p2g<8>(p, a, s) : dispatch_p2g<4>(p, a, s);
}

cudaError_t launch_g2p(ewald_plan_s *p, const void *grid, bool grid_f64, cudaStream_t s)
{
    GridArgs a = grid_args(p);
    a.grid = const_cast<void *>(grid);
    a.scale = 1.0;
    return p->g.T == 8 ? dispatch_g2p<8>(p, a, grid_f64, s) : dispatch_g2p<4>(p, a, grid_f64, s);
}

cudaError_t launch_g2p_scaled(ewald_plan_s *p, const void *grid, bool grid_f64, double scale,
                              cudaStream_t s)
{
    GridArgs a = grid_args(p);
    a.grid = const_cast<void *>(grid);
    a.scale = scale;
    return p->g.T == 8 ? dispatch_g2p<8>(p, a, grid_f64, s) : dispatch_g2p<4>(p, a, grid_f64, s);
}

}  // namespace ewg
