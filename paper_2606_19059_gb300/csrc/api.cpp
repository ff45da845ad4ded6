// api.cpp -- the C ABI of include/ewald_gb300.h: plan lifecycle and the
// apply pipeline of Algorithm 1 (bin, P2P || P2G -> FFT -> CNV -> IFFT -> G2P,
// SUM).  P2P runs on a second stream, concurrently with the far field, as the
// stages are independent until SUM.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

using namespace ewg;

namespace {

const double kPi = 3.14159265358979323846;

#define EW_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            cudaGetLastError();                          \
            return e_ == cudaErrorMemoryAllocation ? EWALD_ENOMEM : EWALD_ECUDA; \
        }                                                \
    } while (0)

#define EW_FFT(call)                                     \
    do {                                                 \
        if ((call) != CUFFT_SUCCESS)                     \
            return EWALD_ECUFFT;                         \
    } while (0)

#define EW_ST(call)                                      \
    do {                                                 \
        ewald_status s_ = (call);                        \
        if (s_ != EWALD_OK)                              \
            return s_;                                   \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
            ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

// Plan workspaces come from one stream-ordered memory pool per device (kept
// reserved: release threshold at its maximum), allocated and freed on the
// plan's own stream: destroying a plan then never waits for the rest of the
// device, as cudaFree would -- a server tearing down one request's plan leaves
// the others running.  Without pool support, plain cudaMalloc/cudaFree.
cudaMemPool_t plan_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    if (dev < 0 || dev >= 64)
        return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        int ok = 0;
        if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess && ok) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t pool = nullptr;
            if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
                pools[dev] = pool;
            }
        }
        cudaGetLastError();
    }
    return pools[dev];
}

// Allocation-failure injection for tests (ewald_debug_fail_alloc): when
// positive, the countdown-th next plan allocation fails as if the device were
// out of memory.  Host state only; no device work is involved.
std::atomic<int> g_fail_alloc_countdown{0};

bool injected_alloc_failure()
{
    int c = g_fail_alloc_countdown.load();
    while (c > 0) {
        if (g_fail_alloc_countdown.compare_exchange_weak(c, c - 1))
            return c == 1;
    }
    return false;
}

template <typename T>
cudaError_t dalloc(ewald_plan_s *p, T **ptr, size_t bytes)
{
    if (injected_alloc_failure())
        return cudaErrorMemoryAllocation;
    if (bytes == 0)
        bytes = 16;
    cudaError_t e;
    if (p->pooled)
        e = cudaMallocFromPoolAsync((void **)ptr, bytes, plan_pool(p->device), p->s2);
    else
        e = cudaMalloc((void **)ptr, bytes);
    if (e == cudaSuccess)
        p->footprint += (int64_t)bytes;
    return e;
}

void dfree(ewald_plan_s *p, void *b)
{
    if (!b)
        return;
    if (p->pooled)
        cudaFreeAsync(b, p->s2);
    else
        cudaFree(b);
}

void free_plan(ewald_plan_s *p)
{
    if (!p)
        return;
    if (p->have_fwd)
        cufftDestroy(p->fwd);
    if (p->have_inv)
        cufftDestroy(p->inv);
    if (p->have_fwd2)
        cufftDestroy(p->fwd2);
    if (p->have_inv2)
        cufftDestroy(p->inv2);
    void *bufs[] = {p->keyn, p->slotn, p->keyt,  p->slott, p->cntn, p->startn, p->cntt,
                    p->startt, p->items, p->item_off, p->permn, p->permt, p->npos, p->nlo, p->nfrc, p->nrec, p->nflo,
                    p->tdat, p->tfrc, p->un, p->uf, p->tab, p->wcoef_dev,
                    p->err, p->hx, p->hf, p->hu, p->fftwork, p->twz, p->wts, p->dl_tf, p->dl_grid, p->dl_spec, p->dl_near};
    for (void *b : bufs)
        dfree(p, b);
    if (!p->ext_grid) {  // a batch's grouped FFT buffers belong to the batch
        dfree(p, p->grid);
        dfree(p, p->spec);
    }
    if (p->own_grid_g2p && p->grid_g2p)
        dfree(p, p->grid_g2p);
    for (auto &g : p->graphs) {
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t e : g.ev)
            if (e)
                cudaEventDestroy(e);
    }
    if (p->s3)
        cudaStreamDestroy(p->s3);
    if (p->s2)
        cudaStreamDestroy(p->s2);
    if (p->ev_fork)
        cudaEventDestroy(p->ev_fork);
    if (p->ev_join)
        cudaEventDestroy(p->ev_join);
    for (auto &e : p->ev)
        if (e)
            cudaEventDestroy(e);
    delete p;
}

ewald_status make_plan(ewald_plan_s *p)
{
    const ewald_params &q = p->prm;
    Geometry &g = p->g;
    g.nc = q.n_c;
    g.cell = q.cell;
    g.K = (int)ceil(q.rc / q.cell - 1e-12);
    if (g.K < 1)
        g.K = 1;
    g.ncells = g.nc * g.nc * g.nc;
    g.nkeys = g.ncells * kSub3;
    g.M = q.M;
    g.P = q.P;
    g.T = q.tile;
    g.nt = g.M / g.T;
    g.ntiles = g.nt * g.nt * g.nt;
    g.KT = (g.P - 1 + g.T - 1) / g.T;
    g.h = q.h;
    g.Mh = g.M / 2 + 1;
    g.nreal = (int64_t)g.M * g.M * g.M;
    g.ncplx = (int64_t)g.M * g.M * g.Mh;
    p->near64 = q.near_f64 != 0;
    p->near_ds = q.near_ds != 0;
    p->ds_r1 = p->near_ds ? ds_split_radius(q.tol, q.xi, q.rc) : 0.0;
    p->fft64 = q.fft_f64 != 0;
    // the double-single grid kernels go with the double-single near field
    p->grid_ds = p->near_ds && grid_ds_supported(g.P, g.T, g.M);

    double werr = 0;
    EW_ST(fit_window(g.P, q.poly_deg, &p->wpoly, &werr));

    // the plan's own stream first: workspaces are allocated on it
    EW_CUDA(cudaStreamCreateWithFlags(&p->s2, cudaStreamNonBlocking));
    EW_CUDA(cudaStreamCreateWithFlags(&p->s3, cudaStreamNonBlocking));
    p->pooled = plan_pool(p->device) != nullptr;

    const int64_t N = p->N;
    const size_t r4 = p->near64 ? 32 : 16, rs = p->near64 ? 8 : 4, fs = p->fft64 ? 8 : 4;
    EW_CUDA(dalloc(p, &p->keyn, 4 * N));
    EW_CUDA(dalloc(p, &p->slotn, 4 * N));
    EW_CUDA(dalloc(p, &p->keyt, 4 * N));
    EW_CUDA(dalloc(p, &p->slott, 4 * N));
    EW_CUDA(dalloc(p, &p->permn, 4 * N));
    EW_CUDA(dalloc(p, &p->permt, 4 * N));
    EW_CUDA(dalloc(p, &p->cntn, 4 * ((size_t)g.nkeys + 1)));
    EW_CUDA(dalloc(p, &p->startn, 4 * ((size_t)g.nkeys + 1)));
    EW_CUDA(dalloc(p, &p->cntt, 4 * ((size_t)g.ntiles + 1)));
    EW_CUDA(dalloc(p, &p->startt, 4 * ((size_t)g.ntiles + 1)));
    EW_CUDA(dalloc(p, &p->items, 4 * ((size_t)g.ncells + 1)));
    EW_CUDA(dalloc(p, &p->item_off, 4 * ((size_t)g.ncells + 1)));
    if (p->near64 && !p->near_ds) {
        EW_CUDA(dalloc(p, &p->npos, r4 * N));
        EW_CUDA(dalloc(p, &p->nfrc, r4 * N));
    } else {
        EW_CUDA(dalloc(p, &p->nrec, 32 * N));
        if (p->near_ds)
            EW_CUDA(dalloc(p, &p->nflo, 16 * N));
    }
    EW_CUDA(dalloc(p, &p->tdat, r4 * N));
    EW_CUDA(dalloc(p, &p->tfrc, r4 * N));
    EW_CUDA(dalloc(p, &p->un, 3 * rs * N));
    EW_CUDA(dalloc(p, &p->uf, 3 * rs * N));
    EW_CUDA(dalloc(p, &p->grid, 3 * fs * (size_t)g.nreal));
    // G2P reads the grid in its own precision: an FP32 copy when the FFT is
    // FP64 and the kernels FP32 (the rounding G2P would apply on each read),
    // a double-single copy for the double-single kernels
    if (p->grid_ds) {
        EW_CUDA(dalloc(p, &p->wts, 4 * 3 * 2 * (size_t)ds_window_stride(g.P) * N));
        EW_CUDA(dalloc(p, &p->grid_g2p, 2 * 3 * 4 * (size_t)g.nreal));
        p->own_grid_g2p = true;
    } else if (!p->near64 && p->fft64) {
        EW_CUDA(dalloc(p, &p->grid_g2p, 3 * 4 * (size_t)g.nreal));
        p->own_grid_g2p = true;
    } else {
        p->grid_g2p = p->grid;
    }
    EW_CUDA(dalloc(p, &p->spec, 3 * 2 * fs * (size_t)g.ncplx));
    EW_CUDA(dalloc(p, &p->tab, fs * (size_t)g.M));
    EW_CUDA(dalloc(p, &p->wcoef_dev, rs * p->wpoly.coef.size()));
    EW_CUDA(dalloc(p, &p->err, sizeof(int)));
    EW_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), p->s2));
    EW_CUDA(cudaMemsetAsync(p->items, 0, 4 * ((size_t)g.ncells + 1), p->s2));
    // binning counters start at zero (each binning's scatter re-zeroes them)
    EW_CUDA(cudaMemsetAsync(p->cntn, 0, 4 * (size_t)g.nkeys, p->s2));
    EW_CUDA(cudaMemsetAsync(p->cntt, 0, 4 * (size_t)g.ntiles, p->s2));
    EW_CUDA(cudaStreamSynchronize(p->s2));  // workspaces ready for any stream

    // window polynomial coefficients in the kernels' precision
    if (p->near64) {
        EW_CUDA(cudaMemcpy(p->wcoef_dev, p->wpoly.coef.data(), 8 * p->wpoly.coef.size(),
                           cudaMemcpyHostToDevice));
    } else {
        std::vector<float> c(p->wpoly.coef.begin(), p->wpoly.coef.end());
        EW_CUDA(cudaMemcpy(p->wcoef_dev, c.data(), 4 * c.size(), cudaMemcpyHostToDevice));
    }
    // CNV table t(n) = e^{-k^2/(4 xi^2)} / w-hat_0(k)^2, zero on the Nyquist plane
    std::vector<double> tab(g.M);
    for (int i = 0; i < g.M; ++i) {
        int n = i <= g.M / 2 ? i : i - g.M;
        if (g.M % 2 == 0 && i == g.M / 2) {
            tab[i] = 0.0;
            continue;
        }
        double k = 2.0 * kPi * n / q.L;
        double wh = kb_window_hat(k, g.h, g.P);
        tab[i] = exp(-k * k / (4.0 * q.xi * q.xi)) / (wh * wh);
    }
    if (p->fft64) {
        EW_CUDA(cudaMemcpy(p->tab, tab.data(), 8 * g.M, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> t(tab.begin(), tab.end());
        EW_CUDA(cudaMemcpy(p->tab, t.data(), 4 * g.M, cudaMemcpyHostToDevice));
    }

    // cuFFT: 3 batched real <-> half-complex transforms of M^3
    int n3[3] = {g.M, g.M, g.M};
    int inembed_r[3] = {g.M, g.M, g.M}, inembed_c[3] = {g.M, g.M, g.Mh};
    // (one work area of our own for both: they never run at the same time)
    size_t wsf = 0, wsi = 0;
    EW_FFT(cufftCreate(&p->fwd));
    p->have_fwd = true;
    EW_FFT(cufftSetAutoAllocation(p->fwd, 0));
    EW_FFT(cufftMakePlanMany(p->fwd, 3, n3, inembed_r, 1, (int)g.nreal, inembed_c, 1,
                             (int)g.ncplx, p->fft64 ? CUFFT_D2Z : CUFFT_R2C, 3, &wsf));
    EW_FFT(cufftCreate(&p->inv));
    p->have_inv = true;
    EW_FFT(cufftSetAutoAllocation(p->inv, 0));
    EW_FFT(cufftMakePlanMany(p->inv, 3, n3, inembed_c, 1, (int)g.ncplx, inembed_r, 1,
                             (int)g.nreal, p->fft64 ? CUFFT_Z2D : CUFFT_C2R, 3, &wsi));
    size_t ws = std::max(wsf, wsi);
    if (fgc_z_supported(g.M)) {
        // FP32: 2-D (y, x) transforms of the 3 M planes, z left to the fused
        // kernel; FP64: 1-D transforms along x of the 3 M^2 rows, y and z
        // left to the double-single kernels
        int n2[2] = {g.M, g.M}, er2[2] = {g.M, g.M}, ec2[2] = {g.M, g.Mh};
        const int rank = p->fft64 ? 1 : 2, batch = p->fft64 ? 3 * g.M * g.M : 3 * g.M;
        const int dr = p->fft64 ? g.M : g.M * g.M, dc = p->fft64 ? g.Mh : g.M * g.Mh;
        int *nn = p->fft64 ? n2 + 1 : n2, *er = p->fft64 ? er2 + 1 : er2, *ec = p->fft64 ? ec2 + 1 : ec2;
        size_t w2f = 0, w2i = 0;
        EW_FFT(cufftCreate(&p->fwd2));
        p->have_fwd2 = true;
        EW_FFT(cufftSetAutoAllocation(p->fwd2, 0));
        EW_FFT(cufftMakePlanMany(p->fwd2, rank, nn, er, 1, dr, ec, 1, dc, p->fft64 ? CUFFT_D2Z : CUFFT_R2C, batch,
                                 &w2f));
        EW_FFT(cufftCreate(&p->inv2));
        p->have_inv2 = true;
        EW_FFT(cufftSetAutoAllocation(p->inv2, 0));
        EW_FFT(cufftMakePlanMany(p->inv2, rank, nn, ec, 1, dc, er, 1, dr, p->fft64 ? CUFFT_Z2D : CUFFT_C2R, batch,
                                 &w2i));
        ws = std::max(ws, std::max(w2f, w2i));
        // w_M^j = e^{-2 pi i j / M}: FP32 (re, im) for k_fgc_z; for the
        // double-single k_fgc_z64 (re h, re l, im h, im l), then the CNV
        // table as (h, l) pairs
        std::vector<float> tw;
        auto hl = [&tw](double v) {
            const float h = (float)v;
            tw.push_back(h);
            tw.push_back((float)(v - (double)h));
        };
        for (int j = 0; j < g.M; ++j) {
            const double c = cos(2.0 * kPi * j / g.M), sn = -sin(2.0 * kPi * j / g.M);
            if (p->fft64) {
                hl(c);
                hl(sn);
            } else {
                tw.push_back((float)c);
                tw.push_back((float)sn);
            }
        }
        if (p->fft64)
            for (int i = 0; i < g.M; ++i)
                hl(tab[i]);
        EW_CUDA(dalloc(p, &p->twz, sizeof(float) * tw.size()));
        EW_CUDA(cudaStreamSynchronize(p->s2));
        EW_CUDA(cudaMemcpy(p->twz, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice));
        p->fgc_fused = true;
    }
    EW_CUDA(dalloc(p, &p->fftwork, ws));
    EW_CUDA(cudaStreamSynchronize(p->s2));
    EW_FFT(cufftSetWorkArea(p->fwd, p->fftwork));
    EW_FFT(cufftSetWorkArea(p->inv, p->fftwork));
    if (p->fgc_fused) {
        EW_FFT(cufftSetWorkArea(p->fwd2, p->fftwork));
        EW_FFT(cufftSetWorkArea(p->inv2, p->fftwork));
    }

    EW_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    EW_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    for (auto &e : p->ev)
        EW_CUDA(cudaEventCreate(&e));
    EW_CUDA(load_p2p_constants());
    p->prm.footprint_bytes = p->footprint;
    return EWALD_OK;
}

// a0: binning of positions (and forces when f != NULL) into both orders.
ewald_status bin(ewald_plan_s *p, const double *x, const double *f, cudaStream_t s)
{
    const Geometry &g = p->g;
    BinArgs a;
    a.x = x;
    a.f = f;
    a.N = p->N;
    a.L = p->prm.L;
    a.cell = g.cell;
    a.h = g.h;
    a.nc = g.nc;
    a.M = g.M;
    a.P = g.P;
    a.T = g.T;
    a.nt = g.nt;
    a.f64 = p->near64;
    a.tf_ds = p->grid_ds;
    // the counters are zero on entry: set at plan creation, and re-zeroed by
    // every binning's scatter once the scans have read them (or here, when a
    // launch of this binning failed)
    cudaError_t e = launch_bin_keys(p, a, s);
    if (e == cudaSuccess)
        e = launch_bin_scans(p, s);
    if (e == cudaSuccess)
        e = launch_bin_scatter(p, a, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaMemsetAsync(p->cntn, 0, 4 * (size_t)g.nkeys, s);
        cudaMemsetAsync(p->cntt, 0, 4 * (size_t)g.ntiles, s);
        return EWALD_ECUDA;
    }
    if (p->grid_ds)
        EW_CUDA(launch_window_ds(p, s));
    p->positions_valid = true;
    return EWALD_OK;
}

void rec(ewald_plan_s *p, int i, cudaStream_t s)
{
    if (p->timing)
        cudaEventRecord(p->ev[i], s);
}

// FFT -> CNV -> IFFT on the plan's grid (in place through the spectrum).
// dl: the double layer's two 3-component grids are transformed too and
// their v-hat added in the CNV (Sec. 2.3).
ewald_status fgc(ewald_plan_s *p, double C, cudaStream_t s, bool dl = false)
{
    if (p->fgc_fused && p->fft64 && !dl) {
        // FP64 spectra: 1-D D2Z along x of the 3 M^2 rows, the y transforms,
        // the z transforms with the CNV and the inverse y transforms in
        // double-single arithmetic, 1-D Z2D along x
        EW_FFT(cufftSetStream(p->fwd2, s));
        EW_FFT(cufftSetStream(p->inv2, s));
        EW_FFT(cufftExecD2Z(p->fwd2, (cufftDoubleReal *)p->grid, (cufftDoubleComplex *)p->spec));
        EW_CUDA(launch_fft_y64(p, false, s));
        rec(p, 3, s);
        EW_CUDA(launch_fgc_z64(p, C, s));
        rec(p, 4, s);
        EW_CUDA(launch_fft_y64(p, true, s));
        EW_FFT(cufftExecZ2D(p->inv2, (cufftDoubleComplex *)p->spec, (cufftDoubleReal *)p->grid));
        rec(p, 5, s);
        return EWALD_OK;
    }
    if (p->fgc_fused && !p->fft64) {
        // 2-D R2C of the 3 M planes (and of the double layer's two density
        // triples), z-FFT + CNV + z-IFFT in one kernel, 2-D C2R
        EW_FFT(cufftSetStream(p->fwd2, s));
        EW_FFT(cufftSetStream(p->inv2, s));
        EW_FFT(cufftExecR2C(p->fwd2, (cufftReal *)p->grid, (cufftComplex *)p->spec));
        for (int t = 0; dl && t < 2; ++t)
            EW_FFT(cufftExecR2C(p->fwd2, (cufftReal *)p->dl_grid + 3 * p->g.nreal * t,
                                (cufftComplex *)p->dl_spec + 3 * p->g.ncplx * t));
        rec(p, 3, s);
        EW_CUDA(dl ? launch_fgc_z_dl(p, C, s) : launch_fgc_z(p, C, s));
        rec(p, 4, s);
        EW_FFT(cufftExecC2R(p->inv2, (cufftComplex *)p->spec, (cufftReal *)p->grid));
        rec(p, 5, s);
        return EWALD_OK;
    }
    EW_FFT(cufftSetStream(p->fwd, s));
    EW_FFT(cufftSetStream(p->inv, s));
    const int ntr = dl ? 3 : 1;
    for (int t = 0; t < ntr; ++t) {
        const int64_t ro = t == 0 ? 0 : 3 * p->g.nreal * (t - 1), co = t == 0 ? 0 : 3 * p->g.ncplx * (t - 1);
        if (p->fft64) {
            cufftDoubleReal *in = t == 0 ? (cufftDoubleReal *)p->grid : (cufftDoubleReal *)p->dl_grid + ro;
            cufftDoubleComplex *out = t == 0 ? (cufftDoubleComplex *)p->spec : (cufftDoubleComplex *)p->dl_spec + co;
            EW_FFT(cufftExecD2Z(p->fwd, in, out));
        } else {
            cufftReal *in = t == 0 ? (cufftReal *)p->grid : (cufftReal *)p->dl_grid + ro;
            cufftComplex *out = t == 0 ? (cufftComplex *)p->spec : (cufftComplex *)p->dl_spec + co;
            EW_FFT(cufftExecR2C(p->fwd, in, out));
        }
    }
    rec(p, 3, s);
    EW_CUDA(launch_scale(p, C, s));
    if (dl)
        EW_CUDA(launch_scale_dl(p, C, s));
    rec(p, 4, s);
    if (p->fft64)
        EW_FFT(cufftExecZ2D(p->inv, (cufftDoubleComplex *)p->spec, (cufftDoubleReal *)p->grid));
    else
        EW_FFT(cufftExecC2R(p->inv, (cufftComplex *)p->spec, (cufftReal *)p->grid));
    rec(p, 5, s);
    return EWALD_OK;
}

// G2P's input from an FP64 grid (the plan's after the inverse FFT, or a
// caller's): the FP32 or double-single copy when the plan keeps one.
cudaError_t prep_g2p_grid(ewald_plan_s *p, const void *grid64, cudaStream_t s)
{
    if (p->grid_ds)
        return launch_grid_split((const double *)grid64, (float *)p->grid_g2p, 3 * p->g.nreal, s);
    if (p->own_grid_g2p)
        return launch_grid_convert(grid64, true, p->grid_g2p, false, 3 * p->g.nreal, s);
    return cudaSuccess;
}

enum Mode { FULL, NEAR_ONLY, FAR_ONLY };

// Everything after binning.  FULL writes u = near + far - self; NEAR_ONLY /
// FAR_ONLY write that stage alone (converted to FP64).
// The double layer's inputs of a combined apply (Sec. 2.3): user-order
// positions and the two source vectors q and n.
struct DlIn {
    const double *x, *q, *n;
};

ewald_status compute(ewald_plan_s *p, const double *f, double *u, Mode mode, cudaStream_t s,
                     const DlIn *dl = nullptr)
{
    const double h3 = p->g.h * p->g.h * p->g.h;
    const double M3 = (double)p->g.nreal;
    const bool overlap = mode == FULL && p->timing != 2;  // timing mode 2: serialised stages
    cudaStream_t sn = overlap ? p->s2 : s;
    // Submission order of the two branches (the block scheduler serves the
    // first-submitted kernel first).  FP32 near field: P2G first, so P2P's
    // single wave runs beside the memory-bound FFTs and the G2P instead of
    // holding every SM's registers while P2G waits (N = 1e5, tol 1e-6: apply
    // 0.673 -> 0.652 ms).  Double-single and FP64 near fields: P2P first --
    // a small double-single P2P launch is latency-bound and the far field
    // submitted before it stretched it (tol 1e-8, N = 1e4: 0.66 -> 1.47 ms).
    const bool far_first = overlap && !p->near_ds && !p->near64;
    // FP32 plans with FP32 FFTs: the double layer's near field in FP32 pairs
    // on the Stokeslet P2P machinery, on the near-field branch
    const bool dl32 = dl && !p->fft64 && !p->near64;
    if (overlap)  // binning done: both branches may start (P2P waits on this)
        EW_CUDA(cudaEventRecord(p->ev_fork, s));
    // P2G of the Stokeslet forces, then of the double layer's six densities
    auto p2g = [&]() -> cudaError_t {
        if (dl && p2g9_supported(p)) {  // all nine components in one pass
            cudaError_t e = launch_dl_densities(p, dl->q, dl->n, s);
            return e == cudaSuccess ? launch_p2g9(p, p->dl_tf, p->dl_grid, s) : e;
        }
        cudaError_t e = launch_p2g(p, s);
        if (e != cudaSuccess || !dl)
            return e;
        const size_t r4 = p->near64 ? sizeof(dvec4) : sizeof(float4);
        const size_t gs = p->fft64 ? sizeof(double) : sizeof(float);
        e = launch_dl_densities(p, dl->q, dl->n, s);
        for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
            // each triple: N quadruples (2 N float4 pairs for double-single grids: same bytes as dvec4)
            const char *src = (const char *)p->dl_tf + t * r4 * p->N;
            char *dst = (char *)p->dl_grid + t * 3 * gs * p->g.nreal;
            e = p->grid_ds ? launch_p2g_ds_with(p, src, (double *)dst, s) : launch_p2g_with(p, src, dst, s);
        }
        return e;
    };
    if (far_first) {
        rec(p, 1, s);
        EW_CUDA(p2g());
        rec(p, 2, s);
    }
    if (mode != FAR_ONLY) {
        if (overlap)
            EW_CUDA(cudaStreamWaitEvent(p->s2, p->ev_fork, 0));
        rec(p, 7, sn);
        EW_CUDA(launch_p2p(p, sn));
        // the double layer's FP32 near field on the same branch, added into
        // the near result before the sum reads it (timed with P2P)
        if (dl && mode == FULL && dl32) {
            EW_CUDA(launch_dl_records(p, dl->q, dl->n, p->dl_near, sn));
            EW_CUDA(launch_p2p_dl32(p, p->dl_near, sn));
        }
        rec(p, 8, sn);
        if (overlap)
            EW_CUDA(cudaEventRecord(p->ev_join, p->s2));
    }
    if (mode != NEAR_ONLY) {
        if (!far_first) {
            rec(p, 1, s);
            EW_CUDA(p2g());
            rec(p, 2, s);
        }
        EW_ST(fgc(p, 8.0 * kPi * h3 / M3, s, dl != nullptr));
        EW_CUDA(prep_g2p_grid(p, p->grid, s));
        EW_CUDA(launch_g2p(p, p->grid_g2p, 1.0, s));
        rec(p, 6, s);
    }
    if (overlap)
        EW_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
    if (mode == FULL) {
        EW_CUDA(launch_sum(p, f, u, s));
        if (dl && !dl32)  // the double layer's FP64 near field, added to u
            EW_CUDA(launch_p2p_dl(p, dl->x, dl->q, dl->n, u, s));
    } else if (mode == NEAR_ONLY) {
        EW_CUDA(launch_copy_out(p->un, p->near64, u, 3 * p->N, s));
    } else {
        EW_CUDA(launch_copy_out(p->uf, p->near64, u, 3 * p->N, s));
    }
    rec(p, 9, s);
    if (p->timing)
        p->timed_once = true;
    return EWALD_OK;
}

bool bad_ptr(const void *a) { return a == nullptr; }

// Repeated applies on the same buffers (an iterative solver's) can run as one
// CUDA graph launch in place of an apply's ~15 launches, copies and memsets.
// Whether that is faster depends on the plan: a replay saves the launch
// overhead but fixes the order in which the near-field and far-field branches
// reach the SMs, and with the persistent double-single P2P launch it measured
// both faster (tol 1e-8, N = 1e4: 0.66 against 1.48 ms) and slower (N = 1e5:
// 5.84 against 5.2 ms; N = 1e6: 58.7 against 49.4 ms).  So each call kind
// measures both on the device and keeps the faster.  The first call with new
// buffers runs directly; the second captures `body` (which enqueues one apply
// on the stream it is given) on the plan's stream s3 and launches the graph on
// the caller's stream between two events; the third runs directly between two
// events; later calls replay until both event pairs have completed (queried,
// never waited on) and then follow the faster.  New buffers start over.  With
// stage timing on, or once a capture has failed, every call runs directly.
template <typename Body>
ewald_status graph_call(ewald_plan_s *p, int kind, const void *a, const void *b, const void *c, cudaStream_t s,
                        Body body)
{
    using Slot = ewald_plan_s::GraphSlot;
    if (p->timing || p->graphs_off)
        return body(s);
    Slot &g = p->graphs[kind];
    if (!(g.a == a && g.b == b && g.c == c)) {
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.a = a;
        g.b = b;
        g.c = c;
        g.calls = 0;
        g.mode = Slot::kUndecided;
    }
    const int call = g.calls < 3 ? g.calls++ : 3;
    if (call == 0 || g.mode == Slot::kDirect)
        return body(s);
    if (call == 1) {
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(p->s3, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        ewald_status st = EWALD_OK;
        if (ok) {
            st = body(p->s3);
            ok = cudaStreamEndCapture(p->s3, &graph) == cudaSuccess && st == EWALD_OK && graph &&
                 cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
        }
        if (graph)
            cudaGraphDestroy(graph);
        for (int k = 0; ok && k < 4; ++k)
            ok = g.ev[k] || cudaEventCreate(&g.ev[k]) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();  // the capture's error, if any, is not the caller's
            if (g.exec)
                cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            p->graphs_off = true;
            return body(s);
        }
        EW_CUDA(cudaGraphUpload(g.exec, s));
        EW_CUDA(cudaEventRecord(g.ev[0], s));
        EW_CUDA(cudaGraphLaunch(g.exec, s));
        EW_CUDA(cudaEventRecord(g.ev[1], s));
        return EWALD_OK;
    }
    if (call == 2) {
        EW_CUDA(cudaEventRecord(g.ev[2], s));
        EW_ST(body(s));
        EW_CUDA(cudaEventRecord(g.ev[3], s));
        return EWALD_OK;
    }
    if (g.mode == Slot::kUndecided) {
        const cudaError_t q1 = cudaEventQuery(g.ev[1]);
        const cudaError_t q3 = q1 == cudaSuccess ? cudaEventQuery(g.ev[3]) : q1;
        if (q3 == cudaErrorNotReady) {
            if (cudaPeekAtLastError() == cudaErrorNotReady)
                cudaGetLastError();  // "not yet" is no error of the caller's
        } else {
            float tg = 0.f, td = 0.f;
            const bool timed = q3 == cudaSuccess && cudaEventElapsedTime(&tg, g.ev[0], g.ev[1]) == cudaSuccess &&
                               cudaEventElapsedTime(&td, g.ev[2], g.ev[3]) == cudaSuccess;
            g.mode = timed && td < tg ? Slot::kDirect : Slot::kGraph;
            if (g.mode == Slot::kDirect) {
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
                return body(s);
            }
        }
    }
    EW_CUDA(cudaGraphLaunch(g.exec, s));
    return EWALD_OK;
}

}  // namespace

// Apply phases for batches of plans (csrc/batch.cpp).
namespace ewg {
ewald_status plan_adopt_grid(ewald_plan_s *p, void *grid, void *spec)
{
    DeviceGuard dg(p->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    EW_CUDA(cudaStreamSynchronize(p->s2));
    const bool alias = p->grid_g2p == p->grid;
    if (!p->ext_grid) {
        dfree(p, p->grid);
        dfree(p, p->spec);
    }
    EW_CUDA(cudaStreamSynchronize(p->s2));
    p->grid = grid;
    p->spec = spec;
    if (alias)
        p->grid_g2p = grid;
    p->ext_grid = true;
    return EWALD_OK;
}

ewald_status plan_set_stream_priority(ewald_plan_s *p, int priority)
{
    DeviceGuard dg(p->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    // the plan's side streams are idle between calls: wait for anything still
    // queued (stream-ordered frees), then replace them
    EW_CUDA(cudaStreamSynchronize(p->s2));
    EW_CUDA(cudaStreamSynchronize(p->s3));
    cudaStream_t a = nullptr, b = nullptr;
    EW_CUDA(cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, priority));
    if (cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, priority) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(a);
        return EWALD_ECUDA;
    }
    cudaStreamDestroy(p->s2);
    cudaStreamDestroy(p->s3);
    p->s2 = a;
    p->s3 = b;
    return EWALD_OK;
}

}  // namespace ewg

extern "C" {

const char *ewald_status_string(ewald_status s)
{
    switch (s) {
    case EWALD_OK: return "ok";
    case EWALD_EINVAL: return "invalid argument";
    case EWALD_ENOMEM: return "out of memory";
    case EWALD_ECUDA: return "CUDA runtime error";
    case EWALD_ECUFFT: return "cuFFT error";
    case EWALD_ETIMEOUT: return "device wait timed out";
    case EWALD_EUNSUPPORTED: return "unsupported parameters";
    }
    return "unknown status";
}

ewald_status ewald_plan_ex(int64_t N, double L, double tol, ewald_dtype dtype,
                           const ewald_params *ov, ewald_plan_t *out)
{
    if (!out)
        return EWALD_EINVAL;
    if (N > (int64_t)INT32_MAX / 4)
        return EWALD_EUNSUPPORTED;
    ewald_params prm;
    EW_ST(choose_params(N, L, tol, dtype, ov, &prm));
    ewald_plan_s *p = new (std::nothrow) ewald_plan_s();
    if (!p)
        return EWALD_ENOMEM;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return EWALD_ECUDA;
    }
    p->N = N;
    p->dtype = dtype;
    p->prm = prm;
    ewald_status st = make_plan(p);
    if (st != EWALD_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return EWALD_OK;
}

ewald_status ewald_plan(int64_t N, double L, double tol, ewald_dtype dtype, ewald_plan_t *out)
{
    return ewald_plan_ex(N, L, tol, dtype, nullptr, out);
}

void ewald_destroy(ewald_plan_t plan)
{
    if (!plan)
        return;
    DeviceGuard dg(plan->device);
    free_plan(plan);
}

ewald_status ewald_get_params(ewald_plan_t plan, ewald_params *out)
{
    if (!plan || !out)
        return EWALD_EINVAL;
    *out = plan->prm;
    return EWALD_OK;
}

ewald_status ewald_apply(ewald_plan_t plan, const double *x, const double *f, double *u,
                         void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(f) || bad_ptr(u))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    return graph_call(plan, 0, x, f, u, (cudaStream_t)stream, [&](cudaStream_t s) -> ewald_status {
        rec(plan, 0, s);
        EW_ST(bin(plan, x, f, s));
        return compute(plan, f, u, FULL, s);
    });
}

ewald_status ewald_set_positions(ewald_plan_t plan, const double *x, void *stream)
{
    if (!plan || bad_ptr(x))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    return bin(plan, x, nullptr, (cudaStream_t)stream);
}

ewald_status ewald_apply_forces(ewald_plan_t plan, const double *f, double *u, void *stream)
{
    if (!plan || bad_ptr(f) || bad_ptr(u))
        return EWALD_EINVAL;
    if (!plan->positions_valid)
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    return graph_call(plan, 1, f, u, nullptr, (cudaStream_t)stream, [&](cudaStream_t s) -> ewald_status {
        rec(plan, 0, s);
        EW_CUDA(launch_gather_forces(plan, f, s));
        return compute(plan, f, u, FULL, s);
    });
}

ewald_status ewald_apply_combined(ewald_plan_t plan, const double *x, const double *f, const double *q,
                                  const double *n, double *u, void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(f) || bad_ptr(q) || bad_ptr(n) || bad_ptr(u))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (!plan->dl_tf) {
        // all four workspaces or none: they are committed to the plan only
        // once every allocation succeeded (dl_tf marks the set as present)
        const size_t r4 = plan->near64 ? sizeof(dvec4) : sizeof(float4);
        const size_t gs = plan->fft64 ? sizeof(double) : sizeof(float);
        void *b[4] = {nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[4] = {2 * r4 * (size_t)plan->N, 2 * 3 * gs * (size_t)plan->g.nreal,
                                 2 * 3 * 2 * gs * (size_t)plan->g.ncplx,
                                 (3 * sizeof(dvec4) + 4 * sizeof(float4)) * (size_t)plan->N};
        const int64_t fp0 = plan->footprint;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = dalloc(plan, &b[k], bytes[k]);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(plan->s2);  // pool allocations ready for `s`
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (void *q : b)
                dfree(plan, q);
            plan->footprint = fp0;
            return e == cudaErrorMemoryAllocation ? EWALD_ENOMEM : EWALD_ECUDA;
        }
        plan->dl_grid = b[1];
        plan->dl_spec = b[2];
        plan->dl_near = b[3];
        plan->dl_tf = b[0];
    }
    rec(plan, 0, s);
    EW_ST(bin(plan, x, f, s));
    const DlIn dl{x, q, n};
    return compute(plan, f, u, FULL, s, &dl);
}

ewald_status ewald_apply_host(ewald_plan_t plan, const double *x_host, const double *f_host,
                              double *u_host, void *stream)
{
    if (!plan || bad_ptr(x_host) || bad_ptr(f_host) || bad_ptr(u_host))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    if (!dg.ok)
        return EWALD_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = 3 * sizeof(double) * (size_t)plan->N;
    // Page-locked buffers have device addresses (unified addressing maps
    // them); over a coherent CPU-GPU link (NVLink-C2C on GB300) the binning
    // kernels then read x and f, and the sum kernel writes u, in place: the
    // bytes cross the link inside those kernels instead of in three staged
    // copies, each with its own start-up latency.
    const void *hp[3] = {x_host, f_host, u_host};
    void *dp[3] = {nullptr, nullptr, nullptr};
    bool pinned = true;
    for (int k = 0; k < 3; ++k) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, hp[k]) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            pinned = false;
        } else {
            dp[k] = at.devicePointer;
        }
    }
    const bool mapped = pinned && dp[0] && dp[1] && dp[2];
    if (!mapped && !plan->hx) {  // device staging for the copies
        EW_CUDA(dalloc(plan, &plan->hx, bytes));
        EW_CUDA(dalloc(plan, &plan->hf, bytes));
        EW_CUDA(dalloc(plan, &plan->hu, bytes));
        EW_CUDA(cudaStreamSynchronize(plan->s2));  // pool allocations ready for `s`
    }
    auto body = [&](cudaStream_t cs) -> ewald_status {
        if (mapped) {
            rec(plan, 0, cs);
            EW_ST(bin(plan, (const double *)dp[0], (const double *)dp[1], cs));
            return compute(plan, (const double *)dp[1], (double *)dp[2], FULL, cs);
        }
        EW_CUDA(cudaMemcpyAsync(plan->hx, x_host, bytes, cudaMemcpyHostToDevice, cs));
        EW_CUDA(cudaMemcpyAsync(plan->hf, f_host, bytes, cudaMemcpyHostToDevice, cs));
        rec(plan, 0, cs);
        EW_ST(bin(plan, plan->hx, plan->hf, cs));
        EW_ST(compute(plan, plan->hf, plan->hu, FULL, cs));
        EW_CUDA(cudaMemcpyAsync(u_host, plan->hu, bytes, cudaMemcpyDeviceToHost, cs));
        return EWALD_OK;
    };
    // graphs only with page-locked host buffers (copies from pageable memory
    // do not capture)
    EW_ST(pinned ? graph_call(plan, 2, x_host, f_host, u_host, s, body) : body(s));
    EW_CUDA(cudaStreamSynchronize(s));
    return EWALD_OK;
}

ewald_status ewald_near_field(ewald_plan_t plan, const double *x, const double *f, double *u,
                              void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(f) || bad_ptr(u))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    rec(plan, 0, s);
    EW_ST(bin(plan, x, f, s));
    return compute(plan, f, u, NEAR_ONLY, s);
}

ewald_status ewald_far_field(ewald_plan_t plan, const double *x, const double *f, double *u,
                             void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(f) || bad_ptr(u))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    rec(plan, 0, s);
    EW_ST(bin(plan, x, f, s));
    return compute(plan, f, u, FAR_ONLY, s);
}

ewald_status ewald_spread(ewald_plan_t plan, const double *x, const double *f, double *grid,
                          void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(f) || bad_ptr(grid))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    EW_ST(bin(plan, x, f, s));
    EW_CUDA(launch_p2g(plan, s));
    EW_CUDA(launch_grid_convert(plan->grid, plan->fft64, grid, true, 3 * plan->g.nreal, s));
    return EWALD_OK;
}

ewald_status ewald_interp(ewald_plan_t plan, const double *x, const double *grid, double *u,
                          void *stream)
{
    if (!plan || bad_ptr(x) || bad_ptr(grid) || bad_ptr(u))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    EW_ST(bin(plan, x, nullptr, s));
    const double h3 = plan->g.h * plan->g.h * plan->g.h;
    const void *g = grid;
    if (!plan->near64 || plan->grid_ds) {  // FP32 kernels: an FP32 copy of the caller's grid
        if (plan->grid_ds)
            EW_CUDA(launch_grid_split(grid, (float *)plan->grid_g2p, 3 * plan->g.nreal, s));
        else
            EW_CUDA(launch_grid_convert(grid, true, plan->grid_g2p, false, 3 * plan->g.nreal, s));
        g = plan->grid_g2p;
    }
    EW_CUDA(launch_g2p(plan, g, h3, s));
    EW_CUDA(launch_copy_out(plan->uf, plan->near64, u, 3 * plan->N, s));
    return EWALD_OK;
}

ewald_status ewald_fourier_convolve(ewald_plan_t plan, const double *grid_in, double *grid_out,
                                    void *stream)
{
    if (!plan || bad_ptr(grid_in) || bad_ptr(grid_out))
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = 3 * plan->g.nreal;
    EW_CUDA(launch_grid_convert(grid_in, true, plan->grid, plan->fft64, n, s));
    EW_ST(fgc(plan, 8.0 * kPi / (double)plan->g.nreal, s));
    EW_CUDA(launch_grid_convert(plan->grid, plan->fft64, grid_out, true, n, s));
    return EWALD_OK;
}

ewald_status ewald_set_timing(ewald_plan_t plan, int enable)
{
    if (!plan || enable < 0 || enable > 2)
        return EWALD_EINVAL;
    plan->timing = enable;
    plan->timed_once = false;
    return EWALD_OK;
}

ewald_status ewald_stage_times(ewald_plan_t plan, ewald_stage_timing *out)
{
    if (!plan || !out)
        return EWALD_EINVAL;
    if (!plan->timed_once)
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    EW_CUDA(cudaEventSynchronize(plan->ev[9]));
    auto el = [&](int a, int b) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, plan->ev[a], plan->ev[b]) != cudaSuccess) {
            cudaGetLastError();
            return 0.0f;
        }
        return ms;
    };
    out->bin_ms = el(0, 7);
    out->p2p_ms = el(7, 8);
    out->p2g_ms = el(1, 2);
    out->fft_ms = el(2, 3);
    out->scale_ms = el(3, 4);
    out->ifft_ms = el(4, 5);
    out->g2p_ms = el(5, 6);
    float t6 = el(0, 6), t8 = el(0, 8), t9 = el(0, 9);
    out->sum_ms = t9 - (t6 > t8 ? t6 : t8);
    out->total_ms = t9;
    return EWALD_OK;
}

ewald_status ewald_sync_status(ewald_plan_t plan, void *stream)
{
    if (!plan)
        return EWALD_EINVAL;
    DeviceGuard dg(plan->device);
    EW_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    EW_CUDA(cudaMemcpy(&flag, plan->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        EW_CUDA(cudaMemset(plan->err, 0, sizeof(int)));
        return EWALD_EINVAL;
    }
    return EWALD_OK;
}

ewald_status ewald_debug_fail_alloc(int32_t nth)
{
    if (nth < 0)
        return EWALD_EINVAL;
    g_fail_alloc_countdown.store(nth);
    return EWALD_OK;
}

ewald_status ewald_launch_counts(ewald_plan_t plan, int32_t *kernels, int32_t *ffts)
{
    if (!plan || !kernels || !ffts)
        return EWALD_EINVAL;
    // bin_keys, the scans (one launch), scatter, p2p, p2g, scale, g2p, sum --
    // plus the FP32 or double-single copy of an FP64 grid, and the
    // double-single window weights
    *kernels = 8 + (plan->own_grid_g2p ? 1 : 0) + (plan->grid_ds ? 1 : 0);
    *ffts = 2;
    return EWALD_OK;
}

}  // extern "C"
