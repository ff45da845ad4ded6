// k_fgc_z64.cu -- steps a3-a5 around the k-space scaling (CNV, eq. (sca)) for
// FP64 spectra (the plans of tol < 1e-6) with M in {64, 128, 256}: the y
// transforms (k_fft_y64), and the z transforms with the CNV of k_fgc_z.cu
// (k_fgc_z64), in double-single arithmetic, between cuFFT's 1-D D2Z and Z2D
// along x of the 3 M^2 rows.
//
// GB300's FP64 pipe runs at 1/64 of its FP32 rate, and cuFFT's FP64
// transforms are bound by it.  Values here are unevaluated sums h + l of two
// FP32 numbers (about 44 significant bits): a complex radix-2 butterfly costs
// ~90 FP32 operations against ~10 FP64 ones, so the z transforms move to the
// FP32 pipe at a fraction of their FP64 time.  The error-free transformations
// are the standard ones (Knuth's two-sum, Dekker's fast two-sum, the FMA
// two-product); the _rn intrinsics keep the compiler from contracting them.
// An FFT in this arithmetic errs by about log2(M) units of 2^-44 of the
// spectrum's norm, far below what the FP64 plans' tolerances need.
//
// A block takes W columns of all three components: phase 1 (a thread per
// (c, n2, w)) loads the column's FP64 values x[R2 n1 + n2], splits them,
// runs the length-R1 DFT and the twiddles w_M^{n2 k1} into shared memory;
// phase 2 (per (c, k1, w)) the length-R2 DFTs, X[c][k1 + R1 k2] in slot
// (c, k2, k1, w); phase 3 (per wave vector and column) the CNV; phase 4 (per
// (c, k1, w)) the inverse length-R2 DFTs and twiddles; phase 5 (per (c, b,
// w)) the inverse length-R1 DFTs, written back as FP64.  The split M = R1 R2,
// the four-step indexing and the CNV are those of k_fgc_z.cu; one thread
// holds one component's column at a time, so that 16-byte values stay within
// a modest register budget.
#include "internal.h"

namespace ewg {
namespace {

struct ds {
    float h, l;
};
struct cds {
    ds re, im;
};

__device__ __forceinline__ ds two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), v = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ ds fast_two_sum(float a, float b)  // |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ds dadd(ds x, ds y)
{
    const ds s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ ds dneg(ds x) { return {-x.h, -x.l}; }
__device__ __forceinline__ ds dsub(ds x, ds y) { return dadd(x, dneg(y)); }
__device__ __forceinline__ ds dmul(ds x, ds y)
{
    const float p = __fmul_rn(x.h, y.h);
    const float e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.h, -p)));
    return fast_two_sum(p, e);
}
// x / y: the FP32 quotient, one correction from the double-single residual
__device__ __forceinline__ ds ddiv(ds x, ds y)
{
    const float q0 = __fdiv_rn(x.h, y.h);
    const ds r = dsub(x, dmul({q0, 0.f}, y));
    return fast_two_sum(q0, __fdiv_rn(r.h, y.h));
}
__device__ __forceinline__ ds split(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double join(ds v) { return (double)v.h + (double)v.l; }

__device__ __forceinline__ cds cadd(cds a, cds b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ cds csub(cds a, cds b) { return {dsub(a.re, b.re), dsub(a.im, b.im)}; }
__device__ __forceinline__ cds cmul(cds a, ds wr, ds wi)  // a (wr + i wi)
{
    return {dsub(dmul(a.re, wr), dmul(a.im, wi)), dadd(dmul(a.re, wi), dmul(a.im, wr))};
}
__device__ __forceinline__ float4 pack(cds a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }
__device__ __forceinline__ cds unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

// cos(2 pi m / 32), m = 0..8, as FP32 high and low parts (h the rounded
// value, l the rounded remainder: h + l within 1e-15), and by the quadrant
// symmetries for every m; folded to immediates once the loops below unroll
__device__ __forceinline__ constexpr float cq_h(int m)
{
    return m == 0   ? 1.f
           : m == 1 ? 0.9807852506637573f
           : m == 2 ? 0.9238795042037964f
           : m == 3 ? 0.8314695954322815f
           : m == 4 ? 0.7071067690849304f
           : m == 5 ? 0.5555702447891235f
           : m == 6 ? 0.3826834261417389f
           : m == 7 ? 0.19509032368659973f
                    : 0.f;
}
__device__ __forceinline__ constexpr float cq_l(int m)
{
    return m == 1   ? 2.9739473106360492e-08f
           : m == 2 ? 2.830748968563057e-08f
           : m == 3 ? 1.687026340846387e-08f
           : m == 4 ? 1.2101617485882343e-08f
           : m == 5 ? -1.1769521357507529e-08f
           : m == 6 ? 6.2233507236442165e-09f
           : m == 7 ? -1.670471427850373e-09f
                    : 0.f;
}
__device__ __forceinline__ constexpr ds cq(int m, float sg) { return {sg * cq_h(m), sg * cq_l(m)}; }
__device__ __forceinline__ constexpr ds cos32(int m)
{
    return m <= 8 ? cq(m, 1.f) : m <= 16 ? cq(16 - m, -1.f) : m <= 24 ? cq(m - 16, -1.f) : cq(32 - m, 1.f);
}
__device__ __forceinline__ constexpr ds sin32(int m) { return cos32((m + 24) & 31); }

__device__ __forceinline__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b)
        r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// in-register DFT of length R in {8, 16}, natural order in and out:
// X[k] = sum_n v[n] e^{-+2 pi i n k / R} (radix-2 decimation in time)
template <int R, bool INV>
__device__ __forceinline__ void dft_ds(cds (&v)[R])
{
    constexpr int B = R == 4 ? 2 : (R == 8 ? 3 : 4);
    static_assert((1 << B) == R, "R is 4, 8 or 16");
    cds t[R];
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
                cds b = t[i + j + len / 2];
                if (m == 8) {  // -+i, exact
                    b = INV ? cds{dneg(b.im), b.re} : cds{b.im, dneg(b.re)};
                } else if (m != 0) {
                    b = cmul(b, cos32(m), INV ? sin32(m) : dneg(sin32(m)));
                }
                const cds a = t[i + j];
                t[i + j] = cadd(a, b);
                t[i + j + len / 2] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
        v[i] = t[i];
}

template <int M>
struct ZSplit64;
template <>
struct ZSplit64<64> {
    static constexpr int R1 = 8, R2 = 8, W = 8;
};
template <>
struct ZSplit64<128> {
    static constexpr int R1 = 16, R2 = 8, W = 4;
};
template <>
struct ZSplit64<256> {
    static constexpr int R1 = 16, R2 = 16, W = 2;
};
constexpr int kZ64Threads = 128;

// spec: [3][M][M][Mh] FP64 complex after the 2-D D2Z of every z plane;
// tw: w_M^j as (re h, re l, im h, im l), j < M; tab: the CNV table split h, l;
// kfac = 2 pi / L, inv4xi2 = 1/(4 xi^2), C as in k_scale (split h, l)
template <int M>
__global__ void __launch_bounds__(kZ64Threads) k_fgc_z64(double2 *__restrict__ spec, const float4 *__restrict__ tw,
                                                         const float2 *__restrict__ tab, float2 kfac2,
                                                         float2 inv4xi22, float2 C2)
{
    constexpr int R1 = ZSplit64<M>::R1, R2 = ZSplit64<M>::R2, W = ZSplit64<M>::W, Mh = M / 2 + 1;
    constexpr int S = R1 * W + W, NT = kZ64Threads;
    static_assert((M * Mh) % W == 0, "the blocks tile the columns");
    __shared__ float4 buf[3 * R2 * S];
    const int64_t plane = (int64_t)M * Mh;
    const int col0 = blockIdx.x * W;
    // phase 1: split, length-R1 DFTs, twiddles w_M^{n2 k1}
    for (int t = threadIdx.x; t < 3 * W * R2; t += NT) {
        const int w = t % W, n2 = (t / W) % R2, c = t / (W * R2);
        const double2 *src = spec + (int64_t)c * M * plane + col0 + w;
        cds v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const double2 x = src[(int64_t)(R2 * n1 + n2) * plane];
            v[n1] = {split(x.x), split(x.y)};
        }
        dft_ds<R1, false>(v);
        float4 *dst = buf + (c * R2 + n2) * S + w;
        dst[0] = pack(v[0]);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            const float4 q = tw[n2 * k1];  // n2 k1 < M
            dst[k1 * W] = pack(cmul(v[k1], {q.x, q.y}, {q.z, q.w}));
        }
    }
    __syncthreads();
    // phase 2: length-R2 DFTs; X[c][k1 + R1 k2] into slot (c, k2, k1, w)
    for (int t = threadIdx.x; t < 3 * W * R1; t += NT) {
        const int w = t % W, k1 = (t / W) % R1, c = t / (W * R1);
        float4 *col = buf + c * R2 * S + k1 * W + w;
        cds v[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2)
            v[n2] = unpack(col[n2 * S]);
        dft_ds<R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            col[k2 * S] = pack(v[k2]);
    }
    __syncthreads();
    // phase 3: the CNV (eq. (sca)) at each wave vector of the block's columns:
    // v-hat = s(k) (|k|^2 phi-hat - k (k . phi-hat)),
    // s(k) = C t(n_x) t(n_y) t(n_z) (1 + |k|^2/(4 xi^2)) / |k|^4, k = 0 dropped
    const ds kfac = {kfac2.x, kfac2.y}, inv4xi2 = {inv4xi22.x, inv4xi22.y}, C = {C2.x, C2.y};
    for (int t = threadIdx.x; t < W * M; t += NT) {
        const int w = t % W, iz = t / W, k1 = iz % R1, k2 = iz / R1;
        float4 *e = buf + k2 * S + k1 * W + w;  // component c at e[c * R2 * S]
        const int colx = col0 + w, ix = colx % Mh, iy = colx / Mh;
        const int ny = iy <= M / 2 ? iy : iy - M, nz = iz <= M / 2 ? iz : iz - M;
        cds o0 = {{0.f, 0.f}, {0.f, 0.f}}, o1 = o0, o2 = o0;
        if (ix != 0 || ny != 0 || nz != 0) {
            // integer multiples of 2 pi / L (the integers exact in FP32)
            const ds kx = dmul(kfac, {(float)ix, 0.f}), ky = dmul(kfac, {(float)ny, 0.f}),
                     kz = dmul(kfac, {(float)nz, 0.f});
            const ds k2s = dadd(dadd(dmul(kx, kx), dmul(ky, ky)), dmul(kz, kz));
            const float2 ta = tab[ix], tb = tab[iy], tc = tab[iz];
            const ds tt = dmul(dmul(dmul(C, {ta.x, ta.y}), dmul({tb.x, tb.y}, {tc.x, tc.y})),
                               dadd({1.f, 0.f}, dmul(k2s, inv4xi2)));
            const ds s = ddiv(tt, dmul(k2s, k2s));
            const cds F0 = unpack(e[0]), F1 = unpack(e[R2 * S]), F2 = unpack(e[2 * R2 * S]);
            const ds dr = dadd(dadd(dmul(kx, F0.re), dmul(ky, F1.re)), dmul(kz, F2.re));
            const ds di = dadd(dadd(dmul(kx, F0.im), dmul(ky, F1.im)), dmul(kz, F2.im));
            o0 = {dmul(s, dsub(dmul(k2s, F0.re), dmul(kx, dr))), dmul(s, dsub(dmul(k2s, F0.im), dmul(kx, di)))};
            o1 = {dmul(s, dsub(dmul(k2s, F1.re), dmul(ky, dr))), dmul(s, dsub(dmul(k2s, F1.im), dmul(ky, di)))};
            o2 = {dmul(s, dsub(dmul(k2s, F2.re), dmul(kz, dr))), dmul(s, dsub(dmul(k2s, F2.im), dmul(kz, di)))};
        }
        e[0] = pack(o0);
        e[R2 * S] = pack(o1);
        e[2 * R2 * S] = pack(o2);
    }
    __syncthreads();
    // phase 4: inverse length-R2 DFTs, twiddles w_M^{-b k1}
    for (int t = threadIdx.x; t < 3 * W * R1; t += NT) {
        const int w = t % W, k1 = (t / W) % R1, c = t / (W * R1);
        float4 *col = buf + c * R2 * S + k1 * W + w;
        cds v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            v[k2] = unpack(col[k2 * S]);
        dft_ds<R2, true>(v);
        col[0] = pack(v[0]);
#pragma unroll
        for (int b = 1; b < R2; ++b) {
            const float4 q = tw[b * k1];  // b k1 < M
            col[b * S] = pack(cmul(v[b], {q.x, q.y}, {-q.z, -q.w}));
        }
    }
    __syncthreads();
    // phase 5: inverse length-R1 DFTs, FP64 values back to the spectrum
    for (int t = threadIdx.x; t < 3 * W * R2; t += NT) {
        const int w = t % W, b = (t / W) % R2, c = t / (W * R2);
        const float4 *src = buf + (c * R2 + b) * S + w;
        cds v[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            v[k1] = unpack(src[k1 * W]);
        dft_ds<R1, true>(v);
        double2 *dst = spec + (int64_t)c * M * plane + col0 + w;
#pragma unroll
        for (int a = 0; a < R1; ++a)
            dst[(int64_t)(R2 * a + b) * plane] = make_double2(join(v[a].re), join(v[a].im));
    }
}

// The y transforms of FP64 spectra in the same arithmetic: after cuFFT's 1-D
// D2Z along x, every (component, z, k_x) column along y goes through the
// length-M DFT (forward) or, after the z kernel, its inverse, so that of the
// three transform directions only the real-to-complex one along x stays on
// the FP64 pipe.  spec: [3 M][M][Mh] (plane, y, k_x); a block takes WY
// consecutive columns (k_x fastest, a block may span two planes).  Forward,
// with y = R2 n1 + n2 and k = k1 + R1 k2: a thread per (n2, column) runs the
// length-R1 DFT and the twiddles into shared memory, a thread per (k1,
// column) the length-R2 DFT and stores X[k1 + R1 k2].  Inverse, with
// y = R2 a + b: a thread per (k1, column) loads X[k1 + R1 k2], runs the
// inverse length-R2 DFT and the twiddles w_M^{-b k1}, a thread per (b,
// column) the inverse length-R1 DFT and stores x[R2 a + b].
template <int M, bool INV>
__global__ void __launch_bounds__(kZ64Threads) k_fft_y64(double2 *__restrict__ spec, const float4 *__restrict__ tw)
{
    constexpr int R1 = ZSplit64<M>::R1, R2 = ZSplit64<M>::R2, WY = 3 * ZSplit64<M>::W, Mh = M / 2 + 1;
    constexpr int S = R1 * WY + WY, NT = kZ64Threads;
    static_assert((3 * M * Mh) % WY == 0, "the blocks tile the columns");
    __shared__ float4 buf[R2 * S];  // slot (n2 or b, k1, w)
    const int colb = blockIdx.x * WY;
    auto column = [&](int w) {  // first element of column colb + w
        const int col = colb + w, pz = col / Mh, kx = col - pz * Mh;
        return spec + (int64_t)pz * M * Mh + kx;
    };
    if (!INV) {
        for (int t = threadIdx.x; t < WY * R2; t += NT) {
            const int w = t % WY, n2 = t / WY;
            const double2 *src = column(w);
            cds v[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) {
                const double2 x = src[(R2 * n1 + n2) * Mh];
                v[n1] = {split(x.x), split(x.y)};
            }
            dft_ds<R1, false>(v);
            float4 *dst = buf + n2 * S + w;
            dst[0] = pack(v[0]);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) {
                const float4 q = tw[n2 * k1];
                dst[k1 * WY] = pack(cmul(v[k1], {q.x, q.y}, {q.z, q.w}));
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < WY * R1; t += NT) {
            const int w = t % WY, k1 = t / WY;
            const float4 *col = buf + k1 * WY + w;
            cds v[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2)
                v[n2] = unpack(col[n2 * S]);
            dft_ds<R2, false>(v);
            double2 *dst = column(w);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2)
                dst[(k1 + R1 * k2) * Mh] = make_double2(join(v[k2].re), join(v[k2].im));
        }
    } else {
        for (int t = threadIdx.x; t < WY * R1; t += NT) {
            const int w = t % WY, k1 = t / WY;
            const double2 *src = column(w);
            cds v[R2];
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const double2 x = src[(k1 + R1 * k2) * Mh];
                v[k2] = {split(x.x), split(x.y)};
            }
            dft_ds<R2, true>(v);
            float4 *col = buf + k1 * WY + w;
            col[0] = pack(v[0]);
#pragma unroll
            for (int b = 1; b < R2; ++b) {
                const float4 q = tw[b * k1];
                col[b * S] = pack(cmul(v[b], {q.x, q.y}, {-q.z, -q.w}));
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < WY * R2; t += NT) {
            const int w = t % WY, b = t / WY;
            const float4 *src = buf + b * S + w;
            cds v[R1];
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                v[k1] = unpack(src[k1 * WY]);
            dft_ds<R1, true>(v);
            double2 *dst = column(w);
#pragma unroll
            for (int a = 0; a < R1; ++a)
                dst[(R2 * a + b) * Mh] = make_double2(join(v[a].re), join(v[a].im));
        }
    }
}

template <int M>
cudaError_t run_fft_y64(ewald_plan_s *p, bool inv, cudaStream_t s)
{
    constexpr int WY = 3 * ZSplit64<M>::W;
    const int nb = 3 * M * (M / 2 + 1) / WY;
    if (inv)
        k_fft_y64<M, true><<<nb, kZ64Threads, 0, s>>>((double2 *)p->spec, (const float4 *)p->twz);
    else
        k_fft_y64<M, false><<<nb, kZ64Threads, 0, s>>>((double2 *)p->spec, (const float4 *)p->twz);
    return cudaGetLastError();
}

float2 split_host(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

template <int M>
cudaError_t run_fgc_z64(ewald_plan_s *p, double C, cudaStream_t s)
{
    const int ncol = M * (M / 2 + 1);
    const float4 *tw = (const float4 *)p->twz;
    const float2 *tab = (const float2 *)(tw + M);
    k_fgc_z64<M><<<ncol / ZSplit64<M>::W, kZ64Threads, 0, s>>>(
        (double2 *)p->spec, tw, tab, split_host(2.0 * 3.14159265358979323846 / p->prm.L),
        split_host(1.0 / (4.0 * p->prm.xi * p->prm.xi)), split_host(C));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fft_y64(ewald_plan_s *p, bool inv, cudaStream_t s)
{
    switch (p->g.M) {
    case 64:
        return run_fft_y64<64>(p, inv, s);
    case 128:
        return run_fft_y64<128>(p, inv, s);
    case 256:
        return run_fft_y64<256>(p, inv, s);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fgc_z64(ewald_plan_s *p, double C, cudaStream_t s)
{
    switch (p->g.M) {
    case 64:
        return run_fgc_z64<64>(p, C, s);
    case 128:
        return run_fgc_z64<128>(p, C, s);
    case 256:
        return run_fgc_z64<256>(p, C, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace ewg
