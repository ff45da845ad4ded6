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
#include <new>
#include <vector>

#include "internal.h"

namespace ewg {
namespace {

template <typename R, typename C2>
__device__ __forceinline__ void scale_elem(C2 *__restrict__ spec, const R *__restrict__ tab, int M, int Mh,
                                           int64_t ncplx, R kfac, R inv4xi2, R C, int64_t idx)
{
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

template <typename R, typename C2>
__global__ void __launch_bounds__(256) k_scale(C2 *__restrict__ spec, const R *__restrict__ tab,
                                               int M, int Mh, int64_t ncplx, R kfac, R inv4xi2, R C)
{
    scale_elem<R, C2>(spec, tab, M, Mh, ncplx, kfac, inv4xi2, C, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// many boxes' CNV in one launch (a block finds its box by binary search)
struct ScaleJob {
    void *spec;
    const void *tab;
    int M, Mh;
    int64_t ncplx;
    double kfac, inv4xi2, C;
};
template <typename R, typename C2>
__global__ void __launch_bounds__(256) k_scale_jobs(const ScaleJob *__restrict__ jobs, const int *__restrict__ base,
                                                    int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const ScaleJob &j = jobs[b];
    scale_elem<R, C2>((C2 *)j.spec, (const R *)j.tab, j.M, j.Mh, j.ncplx, (R)j.kfac, (R)j.inv4xi2, (R)j.C,
                      (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x);
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

struct ScaleBoxes {
    ScaleJob *jobs[2] = {nullptr, nullptr};  // [0] FP32 spectra, [1] FP64
    int *base[2] = {nullptr, nullptr}, n[2] = {0, 0};
    unsigned grid[2] = {0, 0};
};

// The CNV of many plans in one launch per precision; spec[i] is plan i's
// half spectrum (its own or its slice of a grouped FFT's buffer).
cudaError_t scale_boxes_create(ewald_plan_s *const *plans, void *const *spec, int n, ScaleBoxes **out)
{
    ScaleBoxes *b = new (std::nothrow) ScaleBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    std::vector<ScaleJob> jobs[2];
    std::vector<int> base[2] = {std::vector<int>(1, 0), std::vector<int>(1, 0)};
    for (int i = 0; i < n; ++i) {
        ewald_plan_s *p = plans[i];
        const int r = p->fft64 ? 1 : 0;
        const double h3 = p->g.h * p->g.h * p->g.h;
        ScaleJob j;
        j.spec = spec[i];
        j.tab = p->tab;
        j.M = p->g.M;
        j.Mh = p->g.Mh;
        j.ncplx = p->g.ncplx;
        j.kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
        j.inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
        j.C = 8.0 * 3.14159265358979323846 * h3 / (double)p->g.nreal;  // as the plan's own CNV
        jobs[r].push_back(j);
        base[r].push_back(base[r].back() + (int)((j.ncplx + 255) / 256));
    }
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        b->n[r] = (int)jobs[r].size();
        b->grid[r] = (unsigned)base[r].back();
        if (!b->n[r])
            continue;
        e = cudaMalloc(&b->jobs[r], sizeof(ScaleJob) * jobs[r].size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->jobs[r], jobs[r].data(), sizeof(ScaleJob) * jobs[r].size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMalloc(&b->base[r], sizeof(int) * base[r].size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->base[r], base[r].data(), sizeof(int) * base[r].size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        scale_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t scale_boxes_launch(const ScaleBoxes *b, cudaStream_t s, int fft64)
{
    if (!fft64 && b->n[0])
        k_scale_jobs<float, float2><<<b->grid[0], 256, 0, s>>>(b->jobs[0], b->base[0], b->n[0]);
    if (fft64 && b->n[1])
        k_scale_jobs<double, double2><<<b->grid[1], 256, 0, s>>>(b->jobs[1], b->base[1], b->n[1]);
    return cudaGetLastError();
}

int scale_boxes_launches(const ScaleBoxes *b) { return (b->n[0] ? 1 : 0) + (b->n[1] ? 1 : 0); }

void scale_boxes_destroy(ScaleBoxes *b)
{
    if (!b)
        return;
    for (int r = 0; r < 2; ++r) {
        if (b->jobs[r])
            cudaFree(b->jobs[r]);
        if (b->base[r])
            cudaFree(b->base[r]);
    }
    delete b;
}

}  // namespace ewg
