// k_fgc.cu -- step a4: the k-space scaling (CNV) of eq. (sca) on the half
// spectrum (Sec. 3.4: conjugate symmetry halves the work).
//
// For every stored wave vector k = 2 pi n / L (n in FFT order, n_x >= 0):
//   v-hat = C * t(n_x) t(n_y) t(n_z) * (1 + |k|^2/(4 xi^2)) / |k|^4
//           * (|k|^2 phi-hat - k (k . phi-hat)),
// i.e. Ghat^F(k) of eq. (GFk) divided by w-hat(k)^2, with the separable
// factors e^{-k_d^2/(4 xi^2)} / w-hat_0(k_d)^2 in the 1-D table t (zero on the
// Nyquist plane of even M) and C = 8 pi h^3 / M^3 carrying the h^3 of
// eq. (g2p) and the 1/M^3 of the inverse FFT.  k = 0 is dropped.  One pass
// over the three components, read once and written once: HBM bound.
#include "internal.h"

namespace ewg {
namespace {

template <typename R, typename C2>
__global__ void __launch_bounds__(256) k_scale(C2 *__restrict__ spec, const R *__restrict__ tab,
                                               int M, int Mh, int64_t ncplx, R kfac, R inv4xi2, R C)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncplx)
        return;
    int ix = (int)(idx % Mh);
    int iy = (int)((idx / Mh) % M);
    int iz = (int)(idx / ((int64_t)Mh * M));
    int ny = iy <= M / 2 ? iy : iy - M;
    int nz = iz <= M / 2 ? iz : iz - M;
    R kx = kfac * ix, ky = kfac * ny, kz = kfac * nz;
    R k2 = kx * kx + ky * ky + kz * kz;
    C2 F0 = spec[idx], F1 = spec[ncplx + idx], F2 = spec[2 * ncplx + idx];
    R s = (R)0;
    if (k2 > (R)0)
        s = C * tab[ix] * tab[iy] * tab[iz] * ((R)1 + k2 * inv4xi2) / (k2 * k2);
    // k . phi-hat (complex)
    R dr = kx * F0.x + ky * F1.x + kz * F2.x;
    R di = kx * F0.y + ky * F1.y + kz * F2.y;
    C2 o0, o1, o2;
    o0.x = s * (k2 * F0.x - kx * dr);
    o0.y = s * (k2 * F0.y - kx * di);
    o1.x = s * (k2 * F1.x - ky * dr);
    o1.y = s * (k2 * F1.y - ky * di);
    o2.x = s * (k2 * F2.x - kz * dr);
    o2.y = s * (k2 * F2.y - kz * di);
    spec[idx] = o0;
    spec[ncplx + idx] = o1;
    spec[2 * ncplx + idx] = o2;
}

}  // namespace

cudaError_t launch_scale(ewald_plan_s *p, double C, cudaStream_t s)
{
    const double kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
    const double inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
    int64_t n = p->g.ncplx;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (p->fft64)
        k_scale<double, double2><<<nb, 256, 0, s>>>((double2 *)p->spec, (const double *)p->tab,
                                                    p->g.M, p->g.Mh, n, kfac, inv4xi2, C);
    else
        k_scale<float, float2><<<nb, 256, 0, s>>>((float2 *)p->spec, (const float *)p->tab, p->g.M,
                                                  p->g.Mh, n, (float)kfac, (float)inv4xi2,
                                                  (float)C);
    return cudaGetLastError();
}

}  // namespace ewg
