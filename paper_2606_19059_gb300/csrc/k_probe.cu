// k_probe.cu -- measured FP32 and FP64 FMA-pipe peaks of the current device,
// the denominators the ALU-bound stages' rooflines can be read against (the
// HBM and tensor peaks come from a STREAM copy and a cuBLAS GEMM; the FMA
// pipes have no such library measure).
//
// Every thread runs 8 independent FMA chains (enough in flight to cover the
// pipe latency at 8 warps per scheduler), a fixed number of iterations, on
// 4 blocks of 256 threads per SM; the result is stored only under a
// never-true data-dependent condition so the chains are not removed.  Flops =
// 2 x chains x iterations x threads, timed with CUDA events after a warm-up.
#include "internal.h"

namespace ewg {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(R seed, int iters, R *sink)
{
    R a[kChains];
    const R b = seed * (R)0.999, c = seed * (R)1e-3;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        a[k] = seed + (R)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                a[k] = fma(a[k], b, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        s += a[k];
    if (s == (R)-1.2345e30)  // never: keeps the chains alive
        sink[blockIdx.x] = s;
}

template <typename R>
cudaError_t time_chains(int dev, int iters, double *tflops)
{
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int blocks = 4 * sms;
    R *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(R) * blocks);
    if (e != cudaSuccess)
        return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch is a warm-up
        cudaEventRecord(t0);
        k_fma_chains<R><<<blocks, kProbeThreads>>>((R)1.0000001, iters, sink);
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        if (e != cudaSuccess)
            break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best)
            best = ms;
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(sink);
    if (e != cudaSuccess)
        return e;
    const double flops = 2.0 * kChains * 4.0 * iters * (double)blocks * kProbeThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace
}  // namespace ewg

extern "C" ewald_status ewald_probe_fma_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops)
{
    if (!fp32_tflops || !fp64_tflops)
        return EWALD_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return EWALD_ECUDA;
    // ~10 ms of FP32 and of FP64 work at the expected rates
    cudaError_t e = ewg::time_chains<float>(device, 1 << 14, fp32_tflops);
    if (e == cudaSuccess)
        e = ewg::time_chains<double>(device, 1 << 9, fp64_tflops);
    cudaSetDevice(prev);
    return e == cudaSuccess ? EWALD_OK : EWALD_ECUDA;
}
