// batch.cpp -- the measured autotuner and batched (graph-captured) applies
// over many independent boxes.
//
// Parameter choice (Sec. 2.4): every parameter follows from one free choice
// once the error terms of eq. (ese) are held below the tolerance -- the paper
// takes rc and minimises the modelled time T(rc), naming the GPU performance
// models of Sec. 5 as the better T.  Here the free choice is the grid size M
// (xi, rc and n_c follow from it through the planner) together with the grid
// tile T of P2G/G2P, and T(M) is measured on the device rather than modelled:
// every candidate meets the same error bound, so the fastest one wins.
//
// A batch holds one plan per box (each with its own N, L, tol and tuned
// parameters) and device buffers for the boxes' x, f and u.  Every stage runs
// for all boxes at once: one launch per kernel (per kernel instantiation for
// the grid stages, which fix P at compile time), a block finding its box by
// binary search over the boxes' block offsets; the near field of all boxes is
// one persistent launch per P2P variant on a second stream; and the boxes
// that share a grid size and FFT precision keep their grids side by side in
// one buffer, transformed by one batched cuFFT plan.  The first apply
// captures all of it into one CUDA graph; later applies replay the graph with
// one launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "internal.h"

#define TUNE_ST(call)                                    \
    do {                                                 \
        ewald_status s_ = (call);                        \
        if (s_ != EWALD_OK)                              \
            return s_;                                   \
    } while (0)

namespace ewg {
namespace {

bool fft_friendly(int m)
{
    if (m % 2)
        return false;
    for (int p : {2, 3, 5, 7})
        while (m % p == 0)
            m /= p;
    return m == 1;
}

ewald_status candidates(int64_t N, double L, double tol, ewald_dtype dtype, int cap,
                        std::vector<ewald_params> &out)
{
    out.clear();
    if (cap < 1)
        return EWALD_EINVAL;
    ewald_params base;
    TUNE_ST(choose_params(N, L, tol, dtype, nullptr, &base));
    out.push_back(base);
    const int P = base.P, M0 = base.M;
    const int lo = std::max(8, (int)std::floor(0.6 * M0)), hi = (int)std::ceil(1.7 * M0);
    std::vector<int> Ms;
    for (int m = 8 * ((lo + 7) / 8); m <= hi && m <= 1024; m += 8)
        if (fft_friendly(m) && m >= P + 2)
            Ms.push_back(m);
    // at most 6 grid sizes, spread over the range, with T = 8; the other
    // tile only at the model's grid size
    const size_t want = 6, nm = Ms.size() < want ? Ms.size() : want;
    for (size_t im = 0; im <= nm; ++im) {
        const int m = im == nm ? M0 : (Ms.size() <= want ? Ms[im] : Ms[(im * (Ms.size() - 1)) / (want - 1)]);
        for (int T : {8, 4}) {
            if ((im == nm) != (T != base.tile))
                continue;
            if ((int)out.size() >= cap)
                return EWALD_OK;
            ewald_params ov;
            memset(&ov, 0, sizeof(ov));
            ov.M = m;
            ov.P = P;
            ov.tile = T;
            ewald_params q;
            if (choose_params(N, L, tol, dtype, &ov, &q) != EWALD_OK || q.tile != T)
                continue;
            // a double-single plan whose grid kernels would fall back to FP64
            // (4^3 tiles): timed alone such a small box can win, but its FP64
            // P2G/G2P, at 1/64 of the FP32 rate, dominates a batch of them
            if (q.near_ds && !grid_ds_supported(q.P, q.tile, q.M))
                continue;
            bool dup = false;
            for (const ewald_params &c : out)
                dup |= c.M == q.M && c.tile == q.tile && c.P == q.P;
            if (!dup)
                out.push_back(q);
        }
    }
    return EWALD_OK;
}

// Override that reproduces a chosen parameter set for any N.
ewald_params override_of(const ewald_params &q)
{
    ewald_params ov;
    memset(&ov, 0, sizeof(ov));
    ov.M = q.M;
    ov.P = q.P;
    ov.tile = q.tile;
    ov.poly_deg = q.poly_deg;
    return ov;
}

// Seeded uniform points and unit-variance forces for timing (the values do
// not change the work much; the counts per cell do, so points are uniform).
void fill_uniform(std::vector<double> &x, std::vector<double> &f, int64_t N, double L)
{
    uint64_t s = 0x9E3779B97F4A7C15ull ^ (uint64_t)N;
    auto next = [&]() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return (double)(s >> 11) * (1.0 / 9007199254740992.0);
    };
    x.resize(3 * N);
    f.resize(3 * N);
    for (int64_t i = 0; i < 3 * N; ++i) {
        x[i] = L * next();
        f[i] = next() - 0.5;
    }
}

struct TuneKey {
    int64_t N;
    double L, tol;
    int dtype;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(N, L, tol, dtype) < std::tie(o.N, o.L, o.tol, o.dtype);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<ewald_params, double>> g_tune_cache;

ewald_status time_candidate(int64_t N, double L, double tol, ewald_dtype dtype,
                            const ewald_params &q, const double *dx, const double *df, double *du,
                            cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *ms)
{
    ewald_params ov = override_of(q);
    ewald_plan_t p = nullptr;
    TUNE_ST(ewald_plan_ex(N, L, tol, dtype, &ov, &p));
    ewald_status st = EWALD_OK;
    std::vector<float> t;
    for (int it = 0; it < 4 && st == EWALD_OK; ++it) {
        if (it >= 1 && cudaEventRecord(e0, s) != cudaSuccess)
            st = EWALD_ECUDA;
        if (st == EWALD_OK)
            st = ewald_apply(p, dx, df, du, s);
        if (st == EWALD_OK && it >= 1) {
            float v = 0.f;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&v, e0, e1) != cudaSuccess)
                st = EWALD_ECUDA;
            t.push_back(v);
        }
    }
    if (st == EWALD_OK && cudaStreamSynchronize(s) != cudaSuccess)
        st = EWALD_ECUDA;
    ewald_destroy(p);
    if (st != EWALD_OK)
        return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return EWALD_OK;
}

}  // namespace
}  // namespace ewg

using namespace ewg;

// Boxes with the same grid size and FFT precision: their grids and half
// spectra side by side, one batched forward and one inverse cuFFT plan.
struct FftGroup {
    int M = 0;
    bool f64 = false;
    int nb = 0;
    void *grid = nullptr, *spec = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
};

struct ewald_batch_s {
    int device = 0;
    int nbox = 0;
    std::vector<ewald_plan_t> plans;
    std::vector<int64_t> N;
    std::vector<size_t> off;  // per box: offset (in doubles) of its x, f, u in `buf`
    double *buf = nullptr;    // x, f, u of every box: 9 N doubles a box
    std::vector<FftGroup> ffts;
    cudaStream_t cap = nullptr, side = nullptr;  // capture origin (far fields with FP64 FFTs), near field
    cudaStream_t far32 = nullptr;                // far fields with FP32 FFTs
    cudaEvent_t far32_done = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t binned = nullptr;     // every box binned
    cudaEvent_t near_done = nullptr;  // the batched near field finished
    P2PBoxes *near = nullptr;         // one persistent P2P launch per variant
    BinBoxes *bin = nullptr;          // binning and sums
    GridBoxes *grids = nullptr;       // P2G and G2P (FP32 and FP64 grid kernels)
    DsGridBoxes *dsgrids = nullptr;   // the double-single grid stages
    ScaleBoxes *scale = nullptr;      // CNV
    ConvBoxes *conv = nullptr;        // FP64 grids -> FP32 copies for G2P
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(ewald_batch_s *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    for (ewald_plan_t p : b->plans)
        ewald_destroy(p);
    if (b->buf)
        cudaFree(b->buf);
    for (FftGroup &g : b->ffts) {
        if (g.have_fwd)
            cufftDestroy(g.fwd);
        if (g.have_inv)
            cufftDestroy(g.inv);
        if (g.grid)
            cudaFree(g.grid);
        if (g.spec)
            cudaFree(g.spec);
    }
    if (b->cap)
        cudaStreamDestroy(b->cap);
    if (b->side)
        cudaStreamDestroy(b->side);
    if (b->far32)
        cudaStreamDestroy(b->far32);
    for (cudaEvent_t e : {b->fork, b->binned, b->near_done, b->far32_done})
        if (e)
            cudaEventDestroy(e);
    p2p_boxes_destroy(b->near);
    bin_boxes_destroy(b->bin);
    grid_boxes_destroy(b->grids);
    ds_grid_boxes_destroy(b->dsgrids);
    scale_boxes_destroy(b->scale);
    conv_boxes_destroy(b->conv);
    delete b;
}

// Group the boxes' FFTs by (M, precision), move each plan's grid and half
// spectrum into its group's buffer, and build the multi-box launches.
ewald_status setup_stages(ewald_batch_s *b)
{
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (int i = 0; i < b->nbox; ++i)
        groups[{b->plans[i]->g.M, b->plans[i]->fft64 ? 1 : 0}].push_back(i);
    std::vector<void *> grid(b->nbox), spec(b->nbox), g2p(b->nbox);
    for (auto &kv : groups) {
        FftGroup g;
        g.M = kv.first.first;
        g.f64 = kv.first.second != 0;
        g.nb = (int)kv.second.size();
        const ewald_plan_s *p0 = b->plans[kv.second[0]];
        const size_t fs = g.f64 ? 8 : 4;
        const int64_t nreal = p0->g.nreal, ncplx = p0->g.ncplx;
        b->ffts.push_back(g);
        FftGroup &G = b->ffts.back();
        if (cudaMalloc(&G.grid, 3 * fs * (size_t)nreal * G.nb) != cudaSuccess ||
            cudaMalloc(&G.spec, 3 * 2 * fs * (size_t)ncplx * G.nb) != cudaSuccess) {
            cudaGetLastError();
            return EWALD_ENOMEM;
        }
        int n3[3] = {G.M, G.M, G.M}, er[3] = {G.M, G.M, G.M}, ec[3] = {G.M, G.M, G.M / 2 + 1};
        size_t ws = 0;
        if (cufftCreate(&G.fwd) != CUFFT_SUCCESS)
            return EWALD_ECUFFT;
        G.have_fwd = true;
        if (cufftMakePlanMany(G.fwd, 3, n3, er, 1, (int)nreal, ec, 1, (int)ncplx, G.f64 ? CUFFT_D2Z : CUFFT_R2C,
                              3 * G.nb, &ws) != CUFFT_SUCCESS)
            return EWALD_ECUFFT;
        if (cufftCreate(&G.inv) != CUFFT_SUCCESS)
            return EWALD_ECUFFT;
        G.have_inv = true;
        if (cufftMakePlanMany(G.inv, 3, n3, ec, 1, (int)ncplx, er, 1, (int)nreal, G.f64 ? CUFFT_Z2D : CUFFT_C2R,
                              3 * G.nb, &ws) != CUFFT_SUCCESS)
            return EWALD_ECUFFT;
        for (int k = 0; k < G.nb; ++k) {
            const int i = kv.second[k];
            void *gk = (char *)G.grid + 3 * fs * (size_t)nreal * k;
            void *sk = (char *)G.spec + 3 * 2 * fs * (size_t)ncplx * k;
            TUNE_ST(plan_adopt_grid(b->plans[i], gk, sk));
            grid[i] = gk;
            spec[i] = sk;
            g2p[i] = b->plans[i]->grid_g2p;
        }
    }
    std::vector<const double *> xs(b->nbox), fs(b->nbox);
    std::vector<double *> us(b->nbox), grid64(b->nbox);
    std::vector<float *> gds(b->nbox);
    std::vector<const void *> csrc;
    std::vector<void *> cdst;
    std::vector<int64_t> cn;
    for (int i = 0; i < b->nbox; ++i) {
        double *x = b->buf + b->off[i];
        xs[i] = x;
        fs[i] = x + 3 * b->N[i];
        us[i] = x + 6 * b->N[i];
        ewald_plan_s *p = b->plans[i];
        grid64[i] = (double *)grid[i];
        gds[i] = (float *)p->grid_g2p;
        if (p->own_grid_g2p && !p->grid_ds) {  // FP64 FFT, FP32 kernels: G2P reads an FP32 copy
            csrc.push_back(grid[i]);
            cdst.push_back(p->grid_g2p);
            cn.push_back(3 * p->g.nreal);
        }
    }
    if (bin_boxes_create(b->plans.data(), xs.data(), fs.data(), us.data(), b->nbox, &b->bin) != cudaSuccess ||
        grid_boxes_create(b->plans.data(), grid.data(), g2p.data(), b->nbox, &b->grids) != cudaSuccess ||
        ds_grid_boxes_create(b->plans.data(), grid64.data(), gds.data(), b->nbox, &b->dsgrids) != cudaSuccess ||
        scale_boxes_create(b->plans.data(), spec.data(), b->nbox, &b->scale) != cudaSuccess ||
        conv_boxes_create(csrc, cdst, cn, &b->conv) != cudaSuccess) {
        cudaGetLastError();
        return EWALD_ECUDA;
    }
    return EWALD_OK;
}

#define BATCH_CUDA(call)                                 \
    do {                                                 \
        if (st == EWALD_OK && (call) != cudaSuccess)     \
            st = EWALD_ECUDA;                            \
    } while (0)

// Record one batched apply into a graph: binning of every box; then three
// branches side by side -- the near field of every box (persistent P2P
// launches), and the far fields of the boxes with FP64 FFTs and with FP32
// FFTs, each as P2G, the grouped forward FFTs, CNV, the grouped inverse FFTs,
// the G2P grid copies and G2P -- joined before the sums.
ewald_status capture(ewald_batch_s *b)
{
    cudaStream_t s = b->cap;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return EWALD_ECUDA;
    ewald_status st = EWALD_OK;
    BATCH_CUDA(bin_boxes_launch(b->bin, s));
    BATCH_CUDA(ds_grid_boxes_launch(b->dsgrids, 0, s));
    BATCH_CUDA(cudaEventRecord(b->binned, s));
    BATCH_CUDA(cudaStreamWaitEvent(b->side, b->binned, 0));
    BATCH_CUDA(cudaStreamWaitEvent(b->far32, b->binned, 0));
    BATCH_CUDA(p2p_boxes_launch(b->near, b->side));
    BATCH_CUDA(cudaEventRecord(b->near_done, b->side));
    for (int f64 = 1; f64 >= 0 && st == EWALD_OK; --f64) {
        cudaStream_t fs = f64 ? s : b->far32;
        BATCH_CUDA(grid_boxes_launch(b->grids, 0, fs, f64));
        if (f64)
            BATCH_CUDA(ds_grid_boxes_launch(b->dsgrids, 1, fs));
        for (FftGroup &g : b->ffts) {
            if (st != EWALD_OK || g.f64 != (f64 != 0))
                continue;
            if (cufftSetStream(g.fwd, fs) != CUFFT_SUCCESS ||
                (g.f64 ? cufftExecD2Z(g.fwd, (cufftDoubleReal *)g.grid, (cufftDoubleComplex *)g.spec)
                       : cufftExecR2C(g.fwd, (cufftReal *)g.grid, (cufftComplex *)g.spec)) != CUFFT_SUCCESS)
                st = EWALD_ECUFFT;
        }
        BATCH_CUDA(scale_boxes_launch(b->scale, fs, f64));
        for (FftGroup &g : b->ffts) {
            if (st != EWALD_OK || g.f64 != (f64 != 0))
                continue;
            if (cufftSetStream(g.inv, fs) != CUFFT_SUCCESS ||
                (g.f64 ? cufftExecZ2D(g.inv, (cufftDoubleComplex *)g.spec, (cufftDoubleReal *)g.grid)
                       : cufftExecC2R(g.inv, (cufftComplex *)g.spec, (cufftReal *)g.grid)) != CUFFT_SUCCESS)
                st = EWALD_ECUFFT;
        }
        if (f64) {
            BATCH_CUDA(conv_boxes_launch(b->conv, fs));
            BATCH_CUDA(ds_grid_boxes_launch(b->dsgrids, 2, fs));
        }
        BATCH_CUDA(grid_boxes_launch(b->grids, 1, fs, f64));
        if (f64)
            BATCH_CUDA(ds_grid_boxes_launch(b->dsgrids, 3, fs));
    }
    BATCH_CUDA(cudaEventRecord(b->far32_done, b->far32));
    BATCH_CUDA(cudaStreamWaitEvent(s, b->far32_done, 0));
    BATCH_CUDA(cudaStreamWaitEvent(s, b->near_done, 0));
    BATCH_CUDA(sum_boxes_launch(b->bin, s));
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (st == EWALD_OK && ee != cudaSuccess)
        st = EWALD_ECUDA;
    if (st != EWALD_OK) {
        if (g)
            cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return EWALD_ECUDA;
    }
    b->graph = g;
    return EWALD_OK;
}

}  // namespace

extern "C" {

ewald_status ewald_autotune_candidates(int64_t N, double L, double tol, ewald_dtype dtype,
                                       int32_t cap, ewald_params *cands, int32_t *n)
{
    if (!cands || !n || cap < 1)
        return EWALD_EINVAL;
    std::vector<ewald_params> c;
    TUNE_ST(candidates(N, L, tol, dtype, cap, c));
    for (size_t i = 0; i < c.size(); ++i)
        cands[i] = c[i];
    *n = (int32_t)c.size();
    return EWALD_OK;
}

ewald_status ewald_autotune(int64_t N, double L, double tol, ewald_dtype dtype, int32_t mode,
                            ewald_params *out, double *ms)
{
    if (!out || (mode != EWALD_TUNE_MODEL && mode != EWALD_TUNE_MEASURE))
        return EWALD_EINVAL;
    std::vector<ewald_params> c;
    TUNE_ST(candidates(N, L, tol, dtype, 24, c));
    if (mode == EWALD_TUNE_MODEL) {
        *out = c[0];
        if (ms)
            *ms = -1.0;
        return EWALD_OK;
    }
    const TuneKey key{N, L, tol, (int)dtype};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second.first;
            if (ms)
                *ms = it->second.second;
            return EWALD_OK;
        }
    }
    std::vector<double> hx, hf;
    fill_uniform(hx, hf, N, L);
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 9 * (size_t)N) != cudaSuccess) {
        cudaGetLastError();
        return EWALD_ENOMEM;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ewald_status st = EWALD_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemcpy(d, hx.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + 3 * N, hf.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice) != cudaSuccess)
        st = EWALD_ECUDA;
    int best = -1;
    double best_ms = 1e300;
    for (size_t i = 0; i < c.size() && st == EWALD_OK; ++i) {
        double t = 0.0;
        const ewald_status ct =
            time_candidate(N, L, tol, dtype, c[i], d, d + 3 * N, d + 6 * N, s, e0, e1, &t);
        if (ct == EWALD_ENOMEM || ct == EWALD_EUNSUPPORTED)
            continue;  // this candidate does not fit; the others may
        if (ct != EWALD_OK) {
            st = ct;
            break;
        }
        if (t < best_ms) {
            best_ms = t;
            best = (int)i;
        }
    }
    if (s)
        cudaStreamDestroy(s);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(d);
    if (st != EWALD_OK)
        return st;
    if (best < 0)
        return EWALD_ENOMEM;
    // the chosen set re-planned for this N (as a plan would report it)
    ewald_params ov = override_of(c[best]), q;
    TUNE_ST(choose_params(N, L, tol, dtype, &ov, &q));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = {q, best_ms};
    }
    *out = q;
    if (ms)
        *ms = best_ms;
    return EWALD_OK;
}

void ewald_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

ewald_status ewald_batch_create(int32_t nbox, const int64_t *N, const double *L, const double *tol,
                                ewald_dtype dtype, int32_t tune_mode, int32_t nstreams,
                                ewald_batch_t *out)
{
    if (!out || nbox < 1 || !N || !L || !tol || nstreams < 1 || nstreams > 64 ||
        (tune_mode != EWALD_TUNE_MODEL && tune_mode != EWALD_TUNE_MEASURE) ||
        (dtype != EWALD_F64 && dtype != EWALD_F32_BULK))
        return EWALD_EINVAL;
    for (int i = 0; i < nbox; ++i)
        if (N[i] < 1 || !(L[i] > 0) || !std::isfinite(L[i]) || !(tol[i] >= 1e-12 && tol[i] <= 1e-2))
            return EWALD_EINVAL;
    ewald_batch_s *b = new (std::nothrow) ewald_batch_s;
    if (!b)
        return EWALD_ENOMEM;
    b->nbox = nbox;
    cudaGetDevice(&b->device);
    b->N.assign(N, N + nbox);
    b->off.resize(nbox);
    size_t total = 0;
    for (int i = 0; i < nbox; ++i) {
        b->off[i] = total;
        total += 9 * (size_t)N[i];
    }
    ewald_status st = EWALD_OK;
    for (int i = 0; i < nbox && st == EWALD_OK; ++i) {
        ewald_params q;
        // the tuned grid is looked up at the half-octave representative of N
        const int64_t Nb = std::max<int64_t>(
            1, (int64_t)std::llround(std::exp2(std::round(2.0 * std::log2((double)N[i])) / 2.0)));
        st = ewald_autotune(Nb, L[i], tol[i], dtype, tune_mode, &q, nullptr);
        if (st != EWALD_OK)
            break;
        ewald_params ov = override_of(q);
        ewald_plan_t p = nullptr;
        st = ewald_plan_ex(N[i], L[i], tol[i], dtype, &ov, &p);
        if (st == EWALD_OK)
            b->plans.push_back(p);
    }
    if (st == EWALD_OK && cudaMalloc(&b->buf, sizeof(double) * total) != cudaSuccess) {
        cudaGetLastError();
        b->buf = nullptr;
        st = EWALD_ENOMEM;
    }
    if (st == EWALD_OK && cudaMemset(b->buf, 0, sizeof(double) * total) != cudaSuccess)
        st = EWALD_ECUDA;
    (void)nstreams;  // every stage is one launch over all boxes now
    if (st == EWALD_OK && (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaStreamCreateWithFlags(&b->far32, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->far32_done, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->binned, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&b->near_done, cudaEventDisableTiming) != cudaSuccess))
        st = EWALD_ECUDA;
    if (st == EWALD_OK && p2p_boxes_create(b->plans.data(), nbox, &b->near) != cudaSuccess) {
        cudaGetLastError();
        st = EWALD_ECUDA;
    }
    if (st == EWALD_OK)
        st = setup_stages(b);
    if (st == EWALD_OK && cudaDeviceSynchronize() != cudaSuccess)
        st = EWALD_ECUDA;
    if (st != EWALD_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return EWALD_OK;
}

ewald_status ewald_batch_buffers(ewald_batch_t b, int32_t box, double **x, double **f, double **u)
{
    if (!b || box < 0 || box >= b->nbox)
        return EWALD_EINVAL;
    double *p = b->buf + b->off[box];
    const int64_t n3 = 3 * b->N[box];
    if (x)
        *x = p;
    if (f)
        *f = p + n3;
    if (u)
        *u = p + 2 * n3;
    return EWALD_OK;
}

ewald_status ewald_batch_get_params(ewald_batch_t b, int32_t box, ewald_params *out)
{
    if (!b || box < 0 || box >= b->nbox || !out)
        return EWALD_EINVAL;
    return ewald_get_params(b->plans[box], out);
}

ewald_status ewald_batch_plan(ewald_batch_t b, int32_t box, ewald_plan_t *out)
{
    if (!b || box < 0 || box >= b->nbox || !out)
        return EWALD_EINVAL;
    *out = b->plans[box];
    return EWALD_OK;
}

ewald_status ewald_batch_apply(ewald_batch_t b, void *stream)
{
    if (!b)
        return EWALD_EINVAL;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != b->device && cudaSetDevice(b->device) != cudaSuccess)
        return EWALD_ECUDA;
    ewald_status st = EWALD_OK;
    if (!b->exec)
        st = capture(b);
    if (st == EWALD_OK && cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess)
        st = EWALD_ECUDA;
    if (dev != b->device && dev >= 0)
        cudaSetDevice(dev);
    return st;
}

ewald_status ewald_batch_launch_counts(ewald_batch_t b, int32_t *kernels, int32_t *ffts)
{
    if (!b || !kernels || !ffts)
        return EWALD_EINVAL;
    *kernels = bin_boxes_launches(b->bin) + sum_boxes_launches(b->bin) + p2p_boxes_launches(b->near) +
               grid_boxes_launches(b->grids) + ds_grid_boxes_launches(b->dsgrids) +
               scale_boxes_launches(b->scale) + conv_boxes_launches(b->conv);
    *ffts = 2 * (int32_t)b->ffts.size();
    return EWALD_OK;
}

void ewald_batch_destroy(ewald_batch_t b) { free_batch(b); }

}  // extern "C"
