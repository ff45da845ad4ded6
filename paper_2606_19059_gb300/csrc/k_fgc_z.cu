// k_fgc_z.cu -- steps a3-a5 around the k-space scaling (CNV, eq. (sca)) for
// FP32 spectra with M in {64, 128, 256}: the forward FFT along z, the
// CNV and the inverse FFT along z in one kernel, between a 2-D (y, x) R2C and
// a 2-D C2R of cuFFT over the 3 M planes.
//
// The 3-D transform is separable: the 2-D R2C over every (component, z)
// plane leaves phi-hat(z; k_y, k_x), a column along z per stored (k_y, k_x).
// A block takes W consecutive columns (consecutive in memory within each
// plane) of all three components, runs the length-M DFT of each column,
// applies the CNV (its projection mixes the three components, all of them in
// one thread's registers), runs the inverse DFT and writes the columns back:
// the spectrum is read and written once instead of three times (the 3-D
// R2C's z pass, the CNV, the 3-D C2R's z pass).
//
// The length-M DFT is the four-step split M = R1 R2 (phases of k_fgc_z
// below): R2 register DFTs of length R1 per column, the twiddles w_M^{n2 k1}
// from a table, then R1 register DFTs of length R2, and the same in reverse
// for the inverse.  The register DFTs are radix-2 decimation in time,
// unrolled.  FP32 arithmetic and twiddles (the FP64 table rounded), the
// precision of the cuFFT FP32 transforms it replaces.
#include "internal.h"

namespace ewg {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// cos(2 pi m / 32) for m = 0..8, and for every m by the quadrant symmetries;
// folded to immediates once the loops below are unrolled
__device__ __forceinline__ constexpr float cos32q(int m)
{
    return m == 0   ? 1.f
           : m == 1 ? 0.980785280403230449126f
           : m == 2 ? 0.923879532511286756128f
           : m == 3 ? 0.831469612302545237079f
           : m == 4 ? 0.707106781186547524401f
           : m == 5 ? 0.555570233019602224743f
           : m == 6 ? 0.382683432365089771728f
           : m == 7 ? 0.195090322016128267848f
                    : 0.f;
}
__device__ __forceinline__ constexpr float cos32(int m)
{
    return m <= 8 ? cos32q(m) : m <= 16 ? -cos32q(16 - m) : m <= 24 ? -cos32q(m - 16) : cos32q(32 - m);
}
__device__ __forceinline__ constexpr float sin32(int m) { return cos32((m + 24) & 31); }

__device__ __forceinline__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b)
        r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// in-register DFT of length R in {4, 8, 16, 32}, natural order in and out:
// X[k] = sum_n v[n] e^{-+2 pi i n k / R} (radix-2 decimation in time)
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R])
{
    constexpr int B = R == 4 ? 2 : (R == 8 ? 3 : (R == 16 ? 4 : 5));
    static_assert((1 << B) == R, "R is 4, 8, 16 or 32");
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i)
        t[bitrev(i, B)] = v[i];
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
        for (int i = 0; i < R; i += len) {
#pragma unroll
            for (int j = 0; j < len / 2; ++j) {
                const int m = j * (32 / len);  // e^{-+2 pi i j / len} = root m of 32
                float2 b = t[i + j + len / 2];
                if (m == 8) {  // -+i
                    b = INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
                } else if (m != 0) {
                    b = cmul(b, make_float2(cos32(m), INV ? sin32(m) : -sin32(m)));
                }
                const float2 a = t[i + j];
                t[i + j] = cadd(a, b);
                t[i + j + len / 2] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
        v[i] = t[i];
}

// M = R1 R2, the columns W a block takes (three components each) and its
// threads: a thread per (c, n2, w) in phases 1 and 3, per (k1, w) in phase 2
template <int M>
struct ZSplit;
template <>
struct ZSplit<64> {
    static constexpr int R1 = 8, R2 = 8, W = 8, MINB = 3;
};
template <>
struct ZSplit<128> {
    static constexpr int R1 = 16, R2 = 8, W = 8, MINB = 3;
};
template <>
struct ZSplit<256> {
    static constexpr int R1 = 32, R2 = 8, W = 8, MINB = 2;
};

// spec: [3][M][M][Mh] after the 2-D R2C of every (component, z) plane;
// tab: the CNV's 1-D table; tw: w_M^j, j = 0..M-1.
//
// A block takes W consecutive columns of all three components.  With
// z = R2 n1 + n2 and k = k1 + R1 k2 the forward DFT is
//   X[k1 + R1 k2] = sum_{n2} w_{R2}^{n2 k2} w_M^{n2 k1} sum_{n1} x[R2 n1 + n2] w_{R1}^{n1 k1}
// and the inverse, with n = R2 a + b,
//   x[R2 a + b] = sum_{k1} w_{R1}^{-a k1} w_M^{-b k1} sum_{k2} X[k1 + R1 k2] w_{R2}^{-b k2}.
// Phase 1 (a thread per (c, n2, w)): the column's x[R2 n1 + n2] straight from
// global memory, the length-R1 DFT, the twiddles, into shared memory.
// Phase 2 (a thread per (k1, w), all three components): the length-R2 DFTs
// give X[c][k1 + R1 k2] for every k2 in registers, where the CNV mixes the
// components; then the inverse's length-R2 DFTs and twiddles, back into the
// same slots.  Phase 3 (a thread per (c, b, w)): the length-R1 inverse DFT and
// the column's x[R2 a + b] straight to global memory.  Slot (c, n2, k1, w)
// sits at (c R2 + n2) S + k1 W + w with S = R1 W + W: the pad puts the rows a
// warp touches at one k1 on different banks.
template <int M>
constexpr int z_threads()
{
    return 3 * ZSplit<M>::R2 > ZSplit<M>::R1 ? 3 * ZSplit<M>::W * ZSplit<M>::R2 : ZSplit<M>::W * ZSplit<M>::R1;
}

template <int M>
__global__ void __launch_bounds__(z_threads<M>(), ZSplit<M>::MINB)
    k_fgc_z(float2 *__restrict__ spec, const float *__restrict__ tab, const float2 *__restrict__ tw, float kfac,
            float inv4xi2, float C)
{
    constexpr int R1 = ZSplit<M>::R1, R2 = ZSplit<M>::R2, W = ZSplit<M>::W, Mh = M / 2 + 1;
    constexpr int S = R1 * W + W;
    static_assert((M * Mh) % W == 0, "the blocks tile the columns");
    __shared__ float2 buf[3 * R2 * S];
    const int64_t plane = (int64_t)M * Mh;
    const int col0 = blockIdx.x * W;
    const int t = threadIdx.x;
    if (t < 3 * W * R2) {
        const int w = t % W, n2 = (t / W) % R2, c = t / (W * R2);
        const float2 *src = spec + (int64_t)c * M * plane + col0 + w;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
            v[n1] = src[(int64_t)(R2 * n1 + n2) * plane];
        dft_reg<R1, false>(v);
        float2 *dst = buf + (c * R2 + n2) * S + w;
        dst[0] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
            dst[k1 * W] = cmul(v[k1], tw[n2 * k1]);  // w_M^{n2 k1}, n2 k1 < M
    }
    __syncthreads();
    if (t < W * R1) {
        const int w = t % W, k1 = t / W;
        float2 v[3][R2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2)
                v[c][n2] = buf[(c * R2 + n2) * S + k1 * W + w];
            dft_reg<R2, false>(v[c]);
        }
        // CNV (eq. (sca)) at k_z = k1 + R1 k2:
        // v-hat = s(k) (|k|^2 phi-hat - k (k . phi-hat))
        const int colx = col0 + w, ix = colx % Mh, iy = colx / Mh;
        const int ny = iy <= M / 2 ? iy : iy - M;
        const float kx = kfac * ix, ky = kfac * ny, txy = C * tab[ix] * tab[iy];
        const float kxy2 = kx * kx + ky * ky;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            const int iz = k1 + R1 * k2, nz = iz <= M / 2 ? iz : iz - M;
            const float kz = kfac * nz, k2s = kxy2 + kz * kz;
            float s = 0.f;
            if (k2s > 0.f)  // fast division: two ulp, |k|^4 far below 2^126
                s = __fdividef(txy * tab[iz] * (1.f + k2s * inv4xi2), k2s * k2s);
            const float2 F0 = v[0][k2], F1 = v[1][k2], F2 = v[2][k2];
            const float dr = kx * F0.x + ky * F1.x + kz * F2.x;
            const float di = kx * F0.y + ky * F1.y + kz * F2.y;
            v[0][k2] = make_float2(s * (k2s * F0.x - kx * dr), s * (k2s * F0.y - kx * di));
            v[1][k2] = make_float2(s * (k2s * F1.x - ky * dr), s * (k2s * F1.y - ky * di));
            v[2][k2] = make_float2(s * (k2s * F2.x - kz * dr), s * (k2s * F2.y - kz * di));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dft_reg<R2, true>(v[c]);
            float2 *dst = buf + c * R2 * S + k1 * W + w;
            dst[0] = v[c][0];
#pragma unroll
            for (int b = 1; b < R2; ++b) {
                const float2 q = tw[b * k1];  // w_M^{-b k1}, b k1 < M
                dst[b * S] = cmul(v[c][b], make_float2(q.x, -q.y));
            }
        }
    }
    __syncthreads();
    if (t < 3 * W * R2) {
        const int w = t % W, b = (t / W) % R2, c = t / (W * R2);
        const float2 *src = buf + (c * R2 + b) * S + w;
        float2 v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            v[k1] = src[k1 * W];
        dft_reg<R1, true>(v);
        float2 *dst = spec + (int64_t)c * M * plane + col0 + w;
#pragma unroll
        for (int a = 0; a < R1; ++a)
            dst[(int64_t)(R2 * a + b) * plane] = v[a];
    }
}

template <int M>
cudaError_t run_fgc_z(ewald_plan_s *p, double C, cudaStream_t s)
{
    constexpr int W = ZSplit<M>::W, NT = z_threads<M>();
    const int ncol = M * (M / 2 + 1);
    const double kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
    const double inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
    k_fgc_z<M><<<ncol / W, NT, 0, s>>>((float2 *)p->spec, (const float *)p->tab, (const float2 *)p->twz,
                                       (float)kfac, (float)inv4xi2, (float)C);
    return cudaGetLastError();
}

// The combined apply's FGC (Sec. 2.3): the Stokeslet triple and the double
// layer's six density components (S_xx, S_yy, S_zz, then S_xy, S_xz, S_yz)
// go through the forward z DFT; the CNV adds the Stokeslet's v-hat and the
// double layer's, v-hat_j += i s'(k) (2 (S k)_j + k_j (tr S - 2 k.S.k / |k|^2))
// with s'(k) = C t(n_x) t(n_y) t(n_z) (1 + |k|^2/(4 xi^2)) / |k|^2, the form of
// the separate k_scale_dl pass; the three results go through the inverse z
// DFT.  Nine components do not fit one thread's registers, so the length-R2
// DFTs, the CNV and the inverse length-R2 DFTs are three phases over the
// shared slots: five phases, four barriers, a loop over the tasks of each.
template <int M>
struct ZSplitDl;
template <>
struct ZSplitDl<64> {
    static constexpr int R1 = 8, R2 = 8, W = 4;
};
template <>
struct ZSplitDl<128> {
    static constexpr int R1 = 16, R2 = 8, W = 4;
};
template <>
struct ZSplitDl<256> {
    static constexpr int R1 = 32, R2 = 8, W = 2;
};
constexpr int kZDlThreads = 256;

// spec: [3][M][M][Mh] (the Stokeslet triple, in and out); dl: [6][M][M][Mh]
// (the density components), both after the 2-D R2C of every z plane
template <int M>
__global__ void __launch_bounds__(kZDlThreads) k_fgc_z_dl(float2 *__restrict__ spec, const float2 *__restrict__ dl,
                                                          const float *__restrict__ tab,
                                                          const float2 *__restrict__ tw, float kfac,
                                                          float inv4xi2, float C)
{
    constexpr int R1 = ZSplitDl<M>::R1, R2 = ZSplitDl<M>::R2, W = ZSplitDl<M>::W, Mh = M / 2 + 1;
    constexpr int S = R1 * W + W, NT = kZDlThreads;
    static_assert((M * Mh) % W == 0, "the blocks tile the columns");
    __shared__ float2 buf[9 * R2 * S];
    const int64_t plane = (int64_t)M * Mh;
    const int col0 = blockIdx.x * W;
    // phase 1: length-R1 DFTs and twiddles, a task per (c, n2, w)
    for (int t = threadIdx.x; t < 9 * W * R2; t += NT) {
        const int w = t % W, n2 = (t / W) % R2, c = t / (W * R2);
        const float2 *src = (c < 3 ? spec + (int64_t)c * M * plane : dl + (int64_t)(c - 3) * M * plane) + col0 + w;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
            v[n1] = src[(int64_t)(R2 * n1 + n2) * plane];
        dft_reg<R1, false>(v);
        float2 *dst = buf + (c * R2 + n2) * S + w;
        dst[0] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
            dst[k1 * W] = cmul(v[k1], tw[n2 * k1]);
    }
    __syncthreads();
    // phase 2: length-R2 DFTs, a task per (c, k1, w); X[c][k1 + R1 k2] lands
    // in slot (c, k2, k1, w)
    for (int t = threadIdx.x; t < 9 * W * R1; t += NT) {
        const int w = t % W, k1 = (t / W) % R1, c = t / (W * R1);
        float2 *col = buf + c * R2 * S + k1 * W + w;
        float2 v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2)
            v[n2] = col[n2 * S];
        dft_reg<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            col[k2 * S] = v[k2];
    }
    __syncthreads();
    // phase 3: the CNV, a task per (k, w); results into the Stokeslet slots
    for (int t = threadIdx.x; t < W * M; t += NT) {
        const int w = t % W, iz = t / W, k1 = iz % R1, k2 = iz / R1;
        float2 *e = buf + k2 * S + k1 * W + w;  // component c at e[c * R2 * S]
        const int colx = col0 + w, ix = colx % Mh, iy = colx / Mh;
        const int ny = iy <= M / 2 ? iy : iy - M, nz = iz <= M / 2 ? iz : iz - M;
        const float kx = kfac * ix, ky = kfac * ny, kz = kfac * nz;
        const float k2s = kx * kx + ky * ky + kz * kz;
        float2 o0 = make_float2(0.f, 0.f), o1 = o0, o2 = o0;
        if (k2s > 0.f) {
            const float tt = C * tab[ix] * tab[iy] * tab[iz] * (1.f + k2s * inv4xi2);
            const float rk = __fdividef(1.f, k2s);  // two ulp
            const float s = tt * rk * rk, sd = tt * rk;
            const float2 F0 = e[0], F1 = e[R2 * S], F2 = e[2 * R2 * S];
            const float dr = kx * F0.x + ky * F1.x + kz * F2.x;
            const float di = kx * F0.y + ky * F1.y + kz * F2.y;
            o0 = make_float2(s * (k2s * F0.x - kx * dr), s * (k2s * F0.y - kx * di));
            o1 = make_float2(s * (k2s * F1.x - ky * dr), s * (k2s * F1.y - ky * di));
            o2 = make_float2(s * (k2s * F2.x - kz * dr), s * (k2s * F2.y - kz * di));
            const float2 Sxx = e[3 * R2 * S], Syy = e[4 * R2 * S], Szz = e[5 * R2 * S];
            const float2 Sxy = e[6 * R2 * S], Sxz = e[7 * R2 * S], Syz = e[8 * R2 * S];
            // S k, then c = tr S - 2 k.S.k / |k|^2
            const float2 ax = make_float2(Sxx.x * kx + Sxy.x * ky + Sxz.x * kz, Sxx.y * kx + Sxy.y * ky + Sxz.y * kz);
            const float2 ay = make_float2(Sxy.x * kx + Syy.x * ky + Syz.x * kz, Sxy.y * kx + Syy.y * ky + Syz.y * kz);
            const float2 az = make_float2(Sxz.x * kx + Syz.x * ky + Szz.x * kz, Sxz.y * kx + Syz.y * ky + Szz.y * kz);
            const float m2 = -2.f * rk;
            const float cr = fmaf(ax.x * kx + ay.x * ky + az.x * kz, m2, Sxx.x + Syy.x + Szz.x);
            const float ci = fmaf(ax.y * kx + ay.y * ky + az.y * kz, m2, Sxx.y + Syy.y + Szz.y);
            // v += i s' w, w = 2 (S k)_j + k_j c
            const float w0r = fmaf(kx, cr, 2.f * ax.x), w0i = fmaf(kx, ci, 2.f * ax.y);
            const float w1r = fmaf(ky, cr, 2.f * ay.x), w1i = fmaf(ky, ci, 2.f * ay.y);
            const float w2r = fmaf(kz, cr, 2.f * az.x), w2i = fmaf(kz, ci, 2.f * az.y);
            o0 = make_float2(fmaf(-sd, w0i, o0.x), fmaf(sd, w0r, o0.y));
            o1 = make_float2(fmaf(-sd, w1i, o1.x), fmaf(sd, w1r, o1.y));
            o2 = make_float2(fmaf(-sd, w2i, o2.x), fmaf(sd, w2r, o2.y));
        }
        e[0] = o0;
        e[R2 * S] = o1;
        e[2 * R2 * S] = o2;
    }
    __syncthreads();
    // phase 4: inverse length-R2 DFTs and twiddles, a task per (c < 3, k1, w)
    for (int t = threadIdx.x; t < 3 * W * R1; t += NT) {
        const int w = t % W, k1 = (t / W) % R1, c = t / (W * R1);
        float2 *col = buf + c * R2 * S + k1 * W + w;
        float2 v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            v[k2] = col[k2 * S];
        dft_reg<R2, true>(v);
        col[0] = v[0];
#pragma unroll
        for (int b = 1; b < R2; ++b) {
            const float2 q = tw[b * k1];  // w_M^{-b k1}
            col[b * S] = cmul(v[b], make_float2(q.x, -q.y));
        }
    }
    __syncthreads();
    // phase 5: inverse length-R1 DFTs, a task per (c < 3, b, w), to global
    for (int t = threadIdx.x; t < 3 * W * R2; t += NT) {
        const int w = t % W, b = (t / W) % R2, c = t / (W * R2);
        const float2 *src = buf + (c * R2 + b) * S + w;
        float2 v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            v[k1] = src[k1 * W];
        dft_reg<R1, true>(v);
        float2 *dst = spec + (int64_t)c * M * plane + col0 + w;
#pragma unroll
        for (int a = 0; a < R1; ++a)
            dst[(int64_t)(R2 * a + b) * plane] = v[a];
    }
}

template <int M>
cudaError_t run_fgc_z_dl(ewald_plan_s *p, double C, cudaStream_t s)
{
    const int ncol = M * (M / 2 + 1);
    const double kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
    const double inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
    k_fgc_z_dl<M><<<ncol / ZSplitDl<M>::W, kZDlThreads, 0, s>>>((float2 *)p->spec, (const float2 *)p->dl_spec,
                                                              (const float *)p->tab, (const float2 *)p->twz,
                                                              (float)kfac, (float)inv4xi2, (float)C);
    return cudaGetLastError();
}

}  // namespace

bool fgc_z_supported(int M) { return M == 64 || M == 128 || M == 256; }

cudaError_t launch_fgc_z(ewald_plan_s *p, double C, cudaStream_t s)
{
    switch (p->g.M) {
    case 64:
        return run_fgc_z<64>(p, C, s);
    case 128:
        return run_fgc_z<128>(p, C, s);
    case 256:
        return run_fgc_z<256>(p, C, s);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fgc_z_dl(ewald_plan_s *p, double C, cudaStream_t s)
{
    switch (p->g.M) {
    case 64:
        return run_fgc_z_dl<64>(p, C, s);
    case 128:
        return run_fgc_z_dl<128>(p, C, s);
    case 256:
        return run_fgc_z_dl<256>(p, C, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace ewg
