// noalloc.cu -- ewald_near_field_noalloc: the near-field (P2P) apply with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a pre-sized
// memory pool or a custom allocator that owns the whole device, plugins that
// must not touch the allocator of the host application, and code paths that
// must not synchronise the device (cudaMalloc/cudaFree can).  For them this
// entry point keeps its whole workspace (cell keys, counting-sort arrays,
// sorted points and the per-point result) in one file-scope __device__ array
// of fixed size.  Every GPU that loads this library holds that array until
// the process exits.
//
// The array's name seen from host code is only a host-side stand-in, not a
// device address; its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call, and
// passed to the kernels.  That first call on a device should therefore come
// before any stream capture.  All calls share the array and it keeps the last
// call's contents: the counters that must start at zero are cleared on the
// stream at the start of every call, and two calls that overlap on the GPU
// (different streams, or different host threads) race on the array.
#include <math.h>

#include <algorithm>
#include <cmath>

#include "erf_rational.h"
#include "internal.h"

namespace ewg {
namespace {

constexpr int64_t kNoAllocMaxN = 32768;      // points
constexpr int kNoAllocMaxCells = 16 * 16 * 16;  // near cells (n_c <= 16)

// byte offsets of the carve-up, each 256-aligned
constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kI32N = al(4 * kNoAllocMaxN);
constexpr size_t kKeys = al(4 * ((size_t)kNoAllocMaxCells * kSub3 + 1));
constexpr size_t kCells = al(4 * ((size_t)kNoAllocMaxCells + 1));
constexpr size_t kV4N = al(32 * kNoAllocMaxN);   // one 4-vector per point (FP64 size)
constexpr size_t kSmall = 256;
constexpr size_t kOffKeyn = 0;
constexpr size_t kOffSlotn = kOffKeyn + kI32N;
constexpr size_t kOffKeyt = kOffSlotn + kI32N;
constexpr size_t kOffSlott = kOffKeyt + kI32N;
constexpr size_t kOffPermn = kOffSlott + kI32N;
constexpr size_t kOffPermt = kOffPermn + kI32N;
constexpr size_t kOffCntn = kOffPermt + kI32N;
constexpr size_t kOffStartn = kOffCntn + kKeys;
constexpr size_t kOffItems = kOffStartn + kKeys;
constexpr size_t kOffItemOff = kOffItems + kCells;
constexpr size_t kOffCntt = kOffItemOff + kCells;
constexpr size_t kOffStartt = kOffCntt + kSmall;
constexpr size_t kOffErr = kOffStartt + kSmall;
constexpr size_t kOffNpos = kOffErr + kSmall;
constexpr size_t kOffNlo = kOffNpos + kV4N;
constexpr size_t kOffNfrc = kOffNlo + kV4N;
constexpr size_t kOffTdat = kOffNfrc + kV4N;
constexpr size_t kOffTfrc = kOffTdat + kV4N;
constexpr size_t kOffUn = kOffTfrc + kV4N;
constexpr size_t kScratchBytes = kOffUn + al(3 * 8 * kNoAllocMaxN);  // about 7 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

unsigned char *g_scratch_addr[64] = {};

// A NaN or Inf input coordinate raised the binning's error flag: every entry
// of u becomes NaN, so the caller sees it without a status read-back.
__global__ void k_nan_if_flagged(const int *__restrict__ err, double *__restrict__ u, int64_t n)
{
    if (*err == 0)
        return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace
}  // namespace ewg

using namespace ewg;

extern "C" ewald_status ewald_near_field_noalloc(int64_t N, const ewald_params *prm, const double *x,
                                                 const double *f, double *u, void *stream)
{
    if (!prm || !x || !f || !u || N < 1)
        return EWALD_EINVAL;
    if (!(prm->L > 0) || !(prm->xi > 0) || !(prm->rc > 0) || !std::isfinite(prm->L) ||
        !std::isfinite(prm->xi) || !std::isfinite(prm->rc))
        return EWALD_EINVAL;
    if (N > kNoAllocMaxN)
        return EWALD_EUNSUPPORTED;  // the fixed workspace holds at most 32768 points
    const double L = prm->L;
    const int nc = prm->n_c > 0 ? prm->n_c : (int)fmax(1.0, floor(L / prm->rc));
    if (nc < 1 || (int64_t)nc * nc * nc > kNoAllocMaxCells)
        return EWALD_EUNSUPPORTED;  // at most 16 cells per side
    const double cell = L / nc;
    const int K = (int)ceil(prm->rc / cell - 1e-12);
    if (K > 2)
        return EWALD_EUNSUPPORTED;
    if (prm->near_ds && prm->xi * prm->rc > ERFCX_DS_X)
        return EWALD_EUNSUPPORTED;  // beyond the double-single erfcx fit

    // one-time set-up on this device: the array's device address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return EWALD_ECUDA;
    }
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return EWALD_ECUDA;
        }
        g_scratch_addr[dev] = (unsigned char *)ptr;
    }
    unsigned char *base = g_scratch_addr[dev];

    // a plan description on the host stack whose buffers all point into the
    // fixed array (the far-field fields describe one 8^3 tile the binning
    // fills but nothing reads)
    ewald_plan_s pl;
    pl.device = dev;
    pl.N = N;
    // double-single pairs (near_ds) keep FP64 sorted arrays and results, as
    // in a plan; near_ds selects them whatever near_f64 says
    pl.near_ds = prm->near_ds != 0;
    pl.near64 = prm->near_f64 != 0 || pl.near_ds;
    pl.ds_r1 = pl.near_ds ? ds_split_radius(prm->tol, prm->xi, prm->rc) : 0.0;
    pl.fft64 = false;
    pl.prm = *prm;
    pl.prm.n_c = nc;
    pl.prm.cell = cell;
    pl.prm.p2p_block = 128;
    Geometry &g = pl.g;
    g.nc = nc;
    g.K = K < 1 ? 1 : K;
    g.cell = cell;
    g.ncells = nc * nc * nc;
    g.nkeys = g.ncells * kSub3;
    g.M = 8;
    g.P = 2;
    g.T = 8;
    g.nt = 1;
    g.ntiles = 1;
    g.KT = 1;
    g.h = L / 8;
    g.Mh = 5;
    g.nreal = 512;
    g.ncplx = 320;
    pl.keyn = (int32_t *)(base + kOffKeyn);
    pl.slotn = (int32_t *)(base + kOffSlotn);
    pl.keyt = (int32_t *)(base + kOffKeyt);
    pl.slott = (int32_t *)(base + kOffSlott);
    pl.permn = (int32_t *)(base + kOffPermn);
    pl.permt = (int32_t *)(base + kOffPermt);
    pl.cntn = (int32_t *)(base + kOffCntn);
    pl.startn = (int32_t *)(base + kOffStartn);
    pl.items = (int32_t *)(base + kOffItems);
    pl.item_off = (int32_t *)(base + kOffItemOff);
    pl.cntt = (int32_t *)(base + kOffCntt);
    pl.startt = (int32_t *)(base + kOffStartt);
    pl.err = (int *)(base + kOffErr);
    pl.npos = base + kOffNpos;
    pl.nlo = base + kOffNlo;
    pl.nfrc = base + kOffNfrc;
    // FP32 records (32 bytes a point) take the position area, FP64 uses
    // npos; the double-single force low parts (16 bytes a point) take nlo's
    const bool recs = !pl.near64 || pl.near_ds;
    pl.nrec = recs ? base + kOffNpos : nullptr;
    pl.nflo = pl.near_ds ? base + kOffNlo : nullptr;
    pl.tdat = base + kOffTdat;
    pl.tfrc = base + kOffTfrc;
    pl.un = base + kOffUn;

    cudaStream_t s = (cudaStream_t)stream;
    BinArgs a;
    a.x = x;
    a.f = f;
    a.N = N;
    a.L = L;
    a.cell = cell;
    a.h = g.h;
    a.nc = nc;
    a.M = g.M;
    a.P = g.P;
    a.T = g.T;
    a.nt = g.nt;
    a.f64 = pl.near64;
    a.tf_ds = false;
    // clear what the binning accumulates into (the array keeps the last call's contents)
    if (cudaMemsetAsync(pl.cntn, 0, 4 * (size_t)g.nkeys, s) != cudaSuccess ||
        cudaMemsetAsync(pl.cntt, 0, 4 * (size_t)g.ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(pl.err, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return EWALD_ECUDA;
    }
    cudaError_t e = launch_bin_keys(&pl, a, s);
    if (e == cudaSuccess)
        e = launch_scan(pl.cntn, pl.startn, g.nkeys, s);
    if (e == cudaSuccess)
        e = launch_scan(pl.cntt, pl.startt, g.ntiles, s);
    if (e == cudaSuccess)  // the work items from the counts, before the scatter re-zeroes them
        e = launch_cell_items(&pl, s);
    if (e == cudaSuccess)
        e = launch_bin_scatter(&pl, a, s);
    if (e == cudaSuccess)
        e = launch_p2p(&pl, s);
    if (e == cudaSuccess)
        e = launch_copy_out(pl.un, pl.near64, u, 3 * N, s);
    if (e == cudaSuccess) {
        k_nan_if_flagged<<<(unsigned)std::min<int64_t>((3 * N + 255) / 256, 1024), 256, 0, s>>>(pl.err, u, 3 * N);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EWALD_ECUDA;
    }
    return EWALD_OK;
}
