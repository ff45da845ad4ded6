// k_dl.cu -- the double-layer (stresslet) part of the combined single and
// double layer potential of Sec. 2.3: every source carries two vectors q and
// n, and the sum over sources and images of T(x_i - y_j + p) applied to
// q_j (x) n_j is added to the Stokeslet sum.
//
// The paper leaves T and its split T = T^N + T^F to another work.  Here
// T_jlm(r) = -6 r_j r_l r_m / r^5 (the stresslet of the Stokeslet
// I/r + r r^T/r^3), and the split screens T = 2 [d_m G_jl - delta_jl d_m phi
// + delta_jm d_l phi + delta_lm d_j phi] (phi = 1/r) the way eq. (g-near)
// screens G:
//   T^N(r) : D = 2 beta r (r.D.r) + 2 gamma (r tr D + (D + D^T) r),
//     beta  = -3 erfc(xi r)/r^5 - (2 xi/sqrt(pi)) (3/r^4 + 2 xi^2/r^2) e^{-xi^2 r^2},
//     gamma = (2 xi^3/sqrt(pi)) e^{-xi^2 r^2};
//   T-hat^F(k) : D-hat = 8 pi i H(k) [(D-hat + D-hat^T) k + k tr D-hat
//                         - 2 k (k.D-hat.k)/k^2] / k^2,
//     H(k) = (1 + k^2/(4 xi^2)) e^{-k^2/(4 xi^2)} (the Stokeslet's screening).
// Only the symmetric part S of D = q (x) n enters, so the far field spreads
// six components (S_xx, S_yy, S_zz) and (S_xy, S_xz, S_yz) -- two triples
// through the Stokeslet's own P2G kernel and batched FFT -- where the paper
// spreads nine; the CNV adds the double layer's v-hat into the Stokeslet's
// before the one inverse FFT and G2P.  T^F is odd: no self term.
//
// Kernels: k_dl_densities (tile-order S, the P2G input format), k_scale_dl
// (CNV, HBM-bound: 6 complex components in, 3 read-modify-written), and
// k_p2p_dl (near field in FP64, one thread per target in near-sorted order,
// (2K+1)^3 neighbour cells of the plan's cell lists).
#include "internal.h"

namespace ewg {
namespace {

template <typename R4>
__global__ void __launch_bounds__(256) k_dl_densities(const double *__restrict__ q, const double *__restrict__ n,
                                                      const int32_t *__restrict__ permt, int64_t N,
                                                      R4 *__restrict__ sd, R4 *__restrict__ so, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N)
        return;
    const int64_t i = permt[t];
    const double q0 = q[3 * i], q1 = q[3 * i + 1], q2 = q[3 * i + 2];
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    if (!(isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(n0) && isfinite(n1) && isfinite(n2)))
        atomicOr(err, 1);
    R4 a, b;
    a.x = q0 * n0;
    a.y = q1 * n1;
    a.z = q2 * n2;
    a.w = 0;
    b.x = 0.5 * (q0 * n1 + q1 * n0);
    b.y = 0.5 * (q0 * n2 + q2 * n0);
    b.z = 0.5 * (q1 * n2 + q2 * n1);
    b.w = 0;
    sd[t] = a;
    so[t] = b;
}

template <typename R, typename C2>
__device__ __forceinline__ C2 cmad(C2 a, R k, C2 acc)
{
    acc.x = fma(a.x, k, acc.x);
    acc.y = fma(a.y, k, acc.y);
    return acc;
}

// v-hat += C t(kx) t(ky) t(kz) (1 + k^2/(4 xi^2)) / k^2 * i [2 S k + k (tr S - 2 k.S.k / k^2)]
// with t the plan's CNV table (e^{-k^2/(4 xi^2)} / w-hat^2 per axis, 0 on the
// Nyquist plane) and C = 8 pi h^3 / M^3, as the Stokeslet's CNV.
template <typename R, typename C2>
__global__ void __launch_bounds__(256) k_scale_dl(C2 *__restrict__ spec, const C2 *__restrict__ sa,
                                                  const C2 *__restrict__ sb, const R *__restrict__ tab, int M,
                                                  int Mh, int64_t ncplx, R kfac, R inv4xi2, R C)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncplx)
        return;
    const int ix = (int)(idx % Mh);
    const int iy = (int)((idx / Mh) % M);
    const int iz = (int)(idx / ((int64_t)Mh * M));
    const int ny = iy <= M / 2 ? iy : iy - M;
    const int nz = iz <= M / 2 ? iz : iz - M;
    const R kx = kfac * ix, ky = kfac * ny, kz = kfac * nz;
    const R k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 > (R)0))
        return;  // the k = 0 mode stays dropped
    const R s = C * tab[ix] * tab[iy] * tab[iz] * ((R)1 + k2 * inv4xi2) / k2;
    const C2 Sxx = sa[idx], Syy = sa[ncplx + idx], Szz = sa[2 * ncplx + idx];
    const C2 Sxy = sb[idx], Sxz = sb[ncplx + idx], Syz = sb[2 * ncplx + idx];
    C2 z;
    z.x = (R)0;
    z.y = (R)0;
    // S k
    const C2 ax = cmad<R>(Sxz, kz, cmad<R>(Sxy, ky, cmad<R>(Sxx, kx, z)));
    const C2 ay = cmad<R>(Syz, kz, cmad<R>(Syy, ky, cmad<R>(Sxy, kx, z)));
    const C2 az = cmad<R>(Szz, kz, cmad<R>(Syz, ky, cmad<R>(Sxz, kx, z)));
    // c = tr S - 2 k.S.k / k^2
    const C2 kSk = cmad<R>(az, kz, cmad<R>(ay, ky, cmad<R>(ax, kx, z)));
    const R m2 = (R)-2 / k2;
    C2 c;
    c.x = fma(kSk.x, m2, Sxx.x + Syy.x + Szz.x);
    c.y = fma(kSk.y, m2, Sxx.y + Syy.y + Szz.y);
    const C2 a[3] = {ax, ay, az};
    const R kk[3] = {kx, ky, kz};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // w = 2 (S k)_j + k_j c; v = i s w
        const R wx = fma(kk[j], c.x, (R)2 * a[j].x), wy = fma(kk[j], c.y, (R)2 * a[j].y);
        C2 v = spec[j * ncplx + idx];
        v.x = fma(-s, wy, v.x);
        v.y = fma(s, wx, v.y);
        spec[j * ncplx + idx] = v;
    }
}

struct DlNearArgs {
    const double *x, *q, *n;
    const int32_t *permn, *keyn, *startn;
    double *u;
    int64_t N;
    double L, inv_L, xi, rc2;
    int nc, K;
};

__device__ __forceinline__ int floor_div(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

// u_i += sum over sources j and images within rc of T^N(x_i - y_j - p) : S_j,
// one thread per target in near-sorted order (so a warp's targets share cells)
__global__ void __launch_bounds__(128) k_p2p_dl(DlNearArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.N)
        return;
    const int i = a.permn[t];
    const int nc = a.nc, K = a.K;
    const int c = a.keyn[i] / kSub3;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const double xi0 = wrap_coord(a.x[3 * i], a.L, a.inv_L);
    const double xi1 = wrap_coord(a.x[3 * i + 1], a.L, a.inv_L);
    const double xi2 = wrap_coord(a.x[3 * i + 2], a.L, a.inv_L);
    const double xi = a.xi, c_e = 2.0 * xi / 1.7724538509055160273;  // 2 xi / sqrt(pi)
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
    for (int oz = -K; oz <= K; ++oz) {
        const int az = cz + oz, sz = floor_div(az, nc), bz = az - sz * nc;
        for (int oy = -K; oy <= K; ++oy) {
            const int ay = cy + oy, sy = floor_div(ay, nc), by = ay - sy * nc;
            for (int ox = -K; ox <= K; ++ox) {
                const int ax = cx + ox, sx = floor_div(ax, nc), bx = ax - sx * nc;
                const int nb = (bz * nc + by) * nc + bx;
                const int s0 = a.startn[nb * kSub3], s1 = a.startn[(nb + 1) * kSub3];
                // the image of cell nb that sits at (ax, ay, az): sources shifted by L (sx, sy, sz)
                const double b0 = xi0 - a.L * sx, b1 = xi1 - a.L * sy, b2 = xi2 - a.L * sz;
                for (int s = s0; s < s1; ++s) {
                    const int j = a.permn[s];
                    const double r0 = b0 - wrap_coord(a.x[3 * j], a.L, a.inv_L);
                    const double r1 = b1 - wrap_coord(a.x[3 * j + 1], a.L, a.inv_L);
                    const double r2 = b2 - wrap_coord(a.x[3 * j + 2], a.L, a.inv_L);
                    const double rr2 = fma(r0, r0, fma(r1, r1, r2 * r2));
                    if (rr2 > a.rc2 || rr2 == 0.0)
                        continue;
                    const double q0 = a.q[3 * j], q1 = a.q[3 * j + 1], q2 = a.q[3 * j + 2];
                    const double n0 = a.n[3 * j], n1 = a.n[3 * j + 1], n2 = a.n[3 * j + 2];
                    const double qr = fma(q0, r0, fma(q1, r1, q2 * r2));
                    const double nr = fma(n0, r0, fma(n1, r1, n2 * r2));
                    const double qn = fma(q0, n0, fma(q1, n1, q2 * n2));
                    const double rr = sqrt(rr2), inv2 = 1.0 / rr2;
                    const double e = exp(-xi * xi * rr2);
                    const double beta = -3.0 * erfc(xi * rr) * inv2 * inv2 / rr -
                                        c_e * (3.0 * inv2 * inv2 + 2.0 * xi * xi * inv2) * e;
                    const double gamma = c_e * xi * xi * e;
                    // 2 beta r (q.r)(n.r) + 2 gamma (r q.n + q n.r + n q.r)
                    const double br = 2.0 * beta * qr * nr, g2 = 2.0 * gamma;
                    u0 += br * r0 + g2 * (r0 * qn + q0 * nr + n0 * qr);
                    u1 += br * r1 + g2 * (r1 * qn + q1 * nr + n1 * qr);
                    u2 += br * r2 + g2 * (r2 * qn + q2 * nr + n2 * qr);
                }
            }
        }
    }
    a.u[3 * i] += u0;
    a.u[3 * i + 1] += u1;
    a.u[3 * i + 2] += u2;
}

}  // namespace

cudaError_t launch_dl_densities(ewald_plan_s *p, const double *q, const double *n, cudaStream_t s)
{
    const int64_t N = p->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (p->near64) {
        dvec4 *sd = (dvec4 *)p->dl_tf;
        k_dl_densities<dvec4><<<nb, 256, 0, s>>>(q, n, p->permt, N, sd, sd + N, p->err);
    } else {
        float4 *sd = (float4 *)p->dl_tf;
        k_dl_densities<float4><<<nb, 256, 0, s>>>(q, n, p->permt, N, sd, sd + N, p->err);
    }
    return cudaGetLastError();
}

cudaError_t launch_scale_dl(ewald_plan_s *p, double C, cudaStream_t s)
{
    const double kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
    const double inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
    const int64_t n = p->g.ncplx;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (p->fft64) {
        const double2 *sa = (const double2 *)p->dl_spec;
        k_scale_dl<double, double2><<<nb, 256, 0, s>>>((double2 *)p->spec, sa, sa + 3 * n,
                                                       (const double *)p->tab, p->g.M, p->g.Mh, n, kfac,
                                                       inv4xi2, C);
    } else {
        const float2 *sa = (const float2 *)p->dl_spec;
        k_scale_dl<float, float2><<<nb, 256, 0, s>>>((float2 *)p->spec, sa, sa + 3 * n, (const float *)p->tab,
                                                     p->g.M, p->g.Mh, n, (float)kfac, (float)inv4xi2,
                                                     (float)C);
    }
    return cudaGetLastError();
}

cudaError_t launch_p2p_dl(ewald_plan_s *p, const double *x, const double *q, const double *n, double *u,
                          cudaStream_t s)
{
    DlNearArgs a;
    a.x = x;
    a.q = q;
    a.n = n;
    a.permn = p->permn;
    a.keyn = p->keyn;
    a.startn = p->startn;
    a.u = u;
    a.N = p->N;
    a.L = p->prm.L;
    a.inv_L = 1.0 / p->prm.L;
    a.xi = p->prm.xi;
    a.rc2 = p->prm.rc * p->prm.rc;
    a.nc = p->g.nc;
    a.K = p->g.K;
    const unsigned nb = (unsigned)((p->N + 127) / 128);
    k_p2p_dl<<<nb, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ewg
