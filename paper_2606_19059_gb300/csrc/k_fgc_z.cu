// k_fgc_z.cu -- steps a3-a5 around the k-space scaling (CNV, eq. (sca)) for
// FP32 spectra with M in {64, 128, 256}: the forward FFT along z, the
// CNV and the inverse FFT along z in one kernel, between a 2-D (y, x) R2C and
// a 2-D C2R of cuFFT over the 3 M planes.
//
// The 3-D transform is separable: the 2-D R2C over every (component, z)
// plane leaves phi-hat(z; k_y, k_x), a column along z per stored (k_y, k_x).
// A block takes W = 2048 / M consecutive columns (consecutive in memory within
// each plane) of all three components into shared memory (48 KB), runs the
// length-M DFT of each column, applies the CNV (its projection mixes the three
// components, all of them resident), runs the inverse DFT and writes the
// columns back: the spectrum is read and written once instead of three times
// (the 3-D R2C's z pass, the CNV, the 3-D C2R's z pass).
//
// The length-M DFT is the four-step split M = R1 R2: with z = R2 n1 + n2 and
// k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_{n2} w_{R2}^{n2 k2} w_M^{n2 k1} sum_{n1} x[R2 n1 + n2] w_{R1}^{n1 k1},
// w_n = e^{-2 pi i / n} (conjugated for the inverse): R2 register DFTs of
// length R1 per column, the twiddles w_M^{n2 k1} from a table, then R1
// register DFTs of length R2.  The register DFTs are radix-2 decimation in
// time, unrolled.  FP32 arithmetic and twiddles (the FP64 table rounded), the
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
    static constexpr int R1 = 32, R2 = 8, W = 4, MINB = 4;
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
            if (k2s > 0.f)
                s = txy * tab[iz] * (1.f + k2s * inv4xi2) / (k2s * k2s);
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

}  // namespace ewg
