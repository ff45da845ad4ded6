// k_p2p.cu -- step a1: the near-field (P2P) sum of Sec. 2.1,
//
//   u^N_i = sum_j sum_p G^N(x_i - x_j + p) f_j   over 0 < |r| <= rc,
//
// with the Hasimoto kernel of eq. (g-near) written as
//   G^N f = (A - B) f + (A + B) r (r.f) / r^2,
//   A = erfc(xi r) / r,   B = (2 xi / sqrt(pi)) e^{-xi^2 r^2}.
//
// Work decomposition (prior art: the shared-memory 1-D variant of Sec. 3.1):
// one block per chunk of targets of one cell; the sources of the (2K+1)^3
// colleague cells stream through shared memory a block at a time; one thread
// per target keeps its sum in registers.  Positions are cell-local, so the
// colleague offset d * cell both places the source cell and applies the
// periodic wrap, and FP32 differences do not cancel against the box size.
//
// erfc: FP64 uses the paper's rational erf(x)/x (Sec. 4) with
// erfc(x)/x = 1/x - erf(x)/x; FP32 uses a rational erfcx times the
// Gaussian it needs anyway (see fit_erf.py for why).
#include <math.h>

#include "erf_rational.h"
#include "internal.h"

namespace ewg {
namespace {

__constant__ float c_erfcx32[ERFCX_F32_N];
__constant__ double c_erfp64[ERF_RAT_F64_N];
__constant__ double c_erfq64[ERF_RAT_F64_N];

struct P2PArgs {
    const void *npos, *nfrc;
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

// One FP32 pair: accumulate G^N(r) f into (ax, ay, az).
__device__ __forceinline__ void pair_f32(const float4 &t, const float4 &s, const float4 &f,
                                         float rc2, float xi, float nxi2log2e, float c2,
                                         float &ax, float &ay, float &az)
{
    float dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 <= rc2 && r2 > 0.0f) {
        float rinv = rsqrtf(r2);
        float x = xi * (r2 * rinv);
        float tt = fast_rcp(fmaf((float)ERFCX_C32, x, 1.0f));
        float p = c_erfcx32[ERFCX_F32_N - 1];
#pragma unroll
        for (int k = ERFCX_F32_N - 2; k >= 0; --k)
            p = fmaf(p, tt, c_erfcx32[k]);
        float g = tt * p;                      // erfcx(xi r)
        float E = fast_ex2(r2 * nxi2log2e);    // e^{-xi^2 r^2}
        float gr = g * rinv;                   // erfc(xi r) e^{xi^2 r^2} / r
        float amb = E * (gr - c2);             // A - B
        float apb = E * (gr + c2);             // A + B
        float rf = fmaf(dx, f.x, fmaf(dy, f.y, dz * f.z));
        float co = apb * rf * (rinv * rinv);
        ax = fmaf(amb, f.x, fmaf(co, dx, ax));
        ay = fmaf(amb, f.y, fmaf(co, dy, ay));
        az = fmaf(amb, f.z, fmaf(co, dz, az));
    }
}

// One FP64 pair with the paper's erf(x)/x rational (Sec. 4).
__device__ __forceinline__ void pair_f64(const dvec4 &t, const dvec4 &s, const dvec4 &f,
                                         double rc2, double xi, double xi2, double c2,
                                         double &ax, double &ay, double &az)
{
    double dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
    double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    if (r2 <= rc2 && r2 > 0.0) {
        double rinv = rsqrt(r2);
        double x = xi * (r2 * rinv);
        double A;
        if (x < ERF_RAT_X64) {
            double z = fma(x, 2.0 / ERF_RAT_X64, -1.0);
            double P = c_erfp64[ERF_RAT_F64_N - 1], Q = c_erfq64[ERF_RAT_F64_N - 1];
#pragma unroll
            for (int k = ERF_RAT_F64_N - 2; k >= 0; --k) {
                P = fma(P, z, c_erfp64[k]);
                Q = fma(Q, z, c_erfq64[k]);
            }
            A = rinv - xi * (P / Q);           // erfc(x)/r = (1/x - erf(x)/x) xi
        } else {
            A = 0.0;                           // erfc(7) ~ 4e-23
        }
        double E = exp(-xi2 * r2);
        double B = c2 * E;
        double amb = A - B, apb = A + B;
        double rf = fma(dx, f.x, fma(dy, f.y, dz * f.z));
        double co = apb * rf * (rinv * rinv);
        ax = fma(amb, f.x, fma(co, dx, ax));
        ay = fma(amb, f.y, fma(co, dy, ay));
        az = fma(amb, f.z, fma(co, dz, az));
    }
}

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Locate this block's (cell, target range) from the per-cell item offsets.
__device__ __forceinline__ bool find_item(const P2PArgs &a, int &c, int &tb, int &te)
{
    int item = blockIdx.x;
    if (item >= a.item_off[a.ncells])
        return false;
    int lo = 0, hi = a.ncells;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a.item_off[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    c = lo;
    int chunk = item - a.item_off[c];
    int nch = a.item_off[c + 1] - a.item_off[c];
    int t0 = a.startn[c * kSub3], t1 = a.startn[(c + 1) * kSub3];
    int per = (t1 - t0 + nch - 1) / nch;
    tb = t0 + chunk * per;
    te = min(t1, tb + per);
    return true;
}

template <typename R, typename R4>
__global__ void k_p2p(P2PArgs a)
{
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *spos = (R4 *)smem;
    R4 *sfrc = spos + blockDim.x;
    int c, tb, te;
    if (!find_item(a, c, tb, te))
        return;
    const R4 *npos = (const R4 *)a.npos;
    const R4 *nfrc = (const R4 *)a.nfrc;
    int t = tb + threadIdx.x;
    bool active = t < te;
    R4 xt;
    if (active)
        xt = npos[t];
    else
        xt.x = xt.y = xt.z = xt.w = (R)0;
    const R rc2 = (R)(a.rc * a.rc), xi = (R)a.xi;
    const R c2 = (R)(2.0 * a.xi / sqrt(3.14159265358979323846));
    const R aux = sizeof(R) == 4 ? (R)(-a.xi * a.xi * 1.4426950408889634) : (R)(a.xi * a.xi);
    R ux = 0, uy = 0, uz = 0;
    const int nc = a.nc;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    for (int dz = -a.K; dz <= a.K; ++dz)
        for (int dy = -a.K; dy <= a.K; ++dy)
            for (int dx = -a.K; dx <= a.K; ++dx) {
                int nb = (wrap(cz + dz, nc) * nc + wrap(cy + dy, nc)) * nc + wrap(cx + dx, nc);
                int s0 = a.startn[nb * kSub3], s1 = a.startn[(nb + 1) * kSub3];
                const R ox = (R)(dx * a.cell), oy = (R)(dy * a.cell), oz = (R)(dz * a.cell);
                for (int base = s0; base < s1; base += blockDim.x) {
                    __syncthreads();
                    int j = base + threadIdx.x;
                    if (j < s1) {
                        R4 p = npos[j];
                        p.x += ox;
                        p.y += oy;
                        p.z += oz;
                        spos[threadIdx.x] = p;
                        sfrc[threadIdx.x] = nfrc[j];
                    }
                    __syncthreads();
                    int n = min((int)blockDim.x, s1 - base);
                    if (active) {
                        // per-tile partial sums keep FP32 accumulation error low
                        R px = 0, py = 0, pz = 0;
#pragma unroll 4
                        for (int k = 0; k < n; ++k) {
                            if constexpr (sizeof(R) == 4)
                                pair_f32(xt, spos[k], sfrc[k], rc2, xi, aux, c2, px, py, pz);
                            else
                                pair_f64(xt, spos[k], sfrc[k], rc2, xi, aux, c2, px, py, pz);
                        }
                        ux += px;
                        uy += py;
                        uz += pz;
                    }
                }
            }
    if (active) {
        int i = a.permn[t];
        R *un = (R *)a.un;
        un[3 * i] = ux;
        un[3 * i + 1] = uy;
        un[3 * i + 2] = uz;
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
    float c32[ERFCX_F32_N];
    for (int k = 0; k < ERFCX_F32_N; ++k)
        c32[k] = (float)erfcx_f32_c[k];
    cudaError_t e = cudaMemcpyToSymbol(c_erfcx32, c32, sizeof(c32));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_erfp64, erf_rat_f64_p, sizeof(erf_rat_f64_p));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_erfq64, erf_rat_f64_q, sizeof(erf_rat_f64_q));
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        g_const_loaded[dev] = true;
    return e;
}

cudaError_t launch_p2p(ewald_plan_s *p, cudaStream_t s)
{
    cudaError_t e = load_p2p_constants();
    if (e != cudaSuccess)
        return e;
    P2PArgs a;
    a.npos = p->npos;
    a.nfrc = p->nfrc;
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
    int blk = p->prm.p2p_block;
    // upper bound on work items: every cell contributes at most count/blk + 1
    int64_t grid = (int64_t)p->g.ncells + (p->N + blk - 1) / blk + 1;
    if (p->near64) {
        size_t sm = 2 * sizeof(dvec4) * blk;
        k_p2p<double, dvec4><<<(unsigned)grid, blk, sm, s>>>(a);
    } else {
        size_t sm = 2 * sizeof(float4) * blk;
        k_p2p<float, float4><<<(unsigned)grid, blk, sm, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ewg
