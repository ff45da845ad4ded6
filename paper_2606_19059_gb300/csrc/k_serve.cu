// k_serve.cu -- force update between the successive applies of a served
// request, as an iterative solve would issue them (no counterpart in the
// paper; it drives the serving workload):
//
//   f <- f + a n,   n_{i,c} ~ N(0, 1),   then f <- f - mean_i(f)   (re-centred)
//
// n comes from the counter-based generator Philox4x32-10 (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011),
// written here from its published definition: counter (i_lo, i_hi, step, 0)
// -- i the point, step the update's index -- under the key (seed_lo, seed_hi),
// ten rounds.  Outputs c0, c1 give u1, u2 in (0, 1] and the Box-Muller pair
// n_x, n_y = sqrt(-2 ln u1) (cos, sin)(2 pi u2); c2, c3 likewise give n_z (the
// cosine of their pair).
#include <math.h>

#include "internal.h"

namespace ewg {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c[0], hi0 = __umulhi(kPhiloxM0, c[0]);
        const uint32_t lo1 = kPhiloxM1 * c[2], hi1 = __umulhi(kPhiloxM1, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
}

// (0, 1]: (u + 1) / 2^32
__device__ __forceinline__ double unit_open0(uint32_t u) { return ((double)u + 1.0) * (1.0 / 4294967296.0); }

// f += a n (n from point i's counter); the per-component sums of the new f
// accumulate in sums[0..2] (FP64 atomics: the mean is subtracted next, and
// its rounding is far below any tolerance).
__global__ void k_perturb(double *__restrict__ f, int64_t N, double a, uint32_t step, uint64_t seed,
                          double *__restrict__ sums)
{
    __shared__ double part[3][32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (i < N) {
        uint32_t c[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), step, 0u};
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double two_pi = 6.283185307179586476925286766559;
        const double r0 = sqrt(-2.0 * log(unit_open0(c[0]))), t0 = two_pi * unit_open0(c[1]);
        const double r1 = sqrt(-2.0 * log(unit_open0(c[2]))), t1 = two_pi * unit_open0(c[3]);
        const double n[3] = {r0 * cos(t0), r0 * sin(t0), r1 * cos(t1)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = f[3 * i + d] + a * n[d];
            f[3 * i + d] = v[d];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double s = v[d];
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0)
            part[d][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += part[threadIdx.x][w];
        atomicAdd(&sums[threadIdx.x], s);
    }
}

__global__ void k_recentre(double *__restrict__ f, int64_t N, const double *__restrict__ sums)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N)
        return;
    const double inv = 1.0 / (double)N;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        f[3 * i + d] -= sums[d] * inv;
}

}  // namespace

cudaError_t launch_perturb_forces(double *f, int64_t N, double a, uint32_t step, uint64_t seed,
                                  double *sums, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess)
        return e;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    k_perturb<<<blocks, 256, 0, s>>>(f, N, a, step, seed, sums);
    k_recentre<<<blocks, 256, 0, s>>>(f, N, sums);
    return cudaGetLastError();
}

}  // namespace ewg
