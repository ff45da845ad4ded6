// k_bin.cu -- step a0 (binning) and a7 (sum) of the apply, plus small
// conversion kernels.
//
// Binning (Sec. 3, "cell lists"): every point gets two keys,
//   * its near-field cell (width L/n_c >= rc) refined by a 2x2x2 sub-cell, so
//     that P2P targets of one warp are spatially compact, and
//   * the grid tile (T^3 grid points) holding its window anchor, for P2G/G2P.
// A counting sort (atomic slot per key, one scan, one scatter) writes both
// orders as structure-of-vec4 arrays with cell-local coordinates.  Unlike the
// paper's padded cell list, cells are compact (offset array), so clustered
// inputs cost no padding.
#include <math.h>

#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace ewg {
namespace {

struct KeyArgs {
    const double *x, *f;
    int64_t N;
    double L, inv_L, cell, fix_scale;  // fix_scale = 2^62 / L
    long long L_bits;                  // bit pattern of L
    int nc, M, T, nt, ceilP2, odd_P;
    int32_t *keyn, *slotn, *keyt, *slott, *cntn, *cntt, *permn, *permt;
    int ncntn, ncntt;  // lengths of cntn and cntt
    const int32_t *startn, *startt;
    void *npos, *nfrc, *nrec, *nflo, *tdat, *tfrc;
    bool tf_ds;
    int *err;
};

// tile-sorted force of a double-single grid: (h.x, h.y, h.z, 0), (l.x, l.y, l.z, 0)
__device__ __forceinline__ void store_force_ds(float4 *t, double fx, double fy, double fz)
{
    const float hx = (float)fx, hy = (float)fy, hz = (float)fz;
    t[0] = make_float4(hx, hy, hz, 0.f);
    t[1] = make_float4((float)(fx - (double)hx), (float)(fy - (double)hy), (float)(fz - (double)hz), 0.f);
}

// A point's bins, computed in fixed point: the wrapped coordinate as
// X = floor(x 2^62 / L) (two FP64 operations a coordinate; everything after
// them is integer arithmetic, GB300's FP64 rate being 1/64 of its FP32 rate).
// With A = 4 X (the box as [0, 2^64)), the near cell is the high word of
// A n_c and the position within it the low word (a fraction times 2^64); the
// grid coordinate x/h + (P odd)/2 is A M (+ 2^63) likewise.
struct Bin {
    uint64_t fc[3];    // position within the near cell, times 2^64
    uint64_t fg[3];    // fractional grid offset delta of the anchor, times 2^64
    int c[3], s[3];    // near cell and sub-cell
    int a[3], tl[3];   // window anchor (wrapped) and its tile
    bool bad;
};

__device__ __forceinline__ Bin compute_bin(const KeyArgs &k, int64_t i)
{
    Bin b;
    b.bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double v = k.x[3 * i + d];
        long long vb = __double_as_longlong(v);
        if (((vb >> 52) & 0x7FF) == 0x7FF) {  // Inf or NaN
            b.bad = true;
            v = 0.0;
            vb = 0;
        }
        // wrap into [0, L) unless already inside (a test on the bit pattern:
        // non-negative doubles order as their bits)
        if (!(vb >= 0 && vb < k.L_bits))
            v = wrap_coord(v, k.L, k.inv_L);
        const uint64_t X = min(__double2ull_rz(v * k.fix_scale), (1ull << 62) - 1ull);
        const uint64_t A = X << 2;
        const int ci = (int)__umul64hi(A, (uint64_t)k.nc);  // <= nc - 1 as A < 2^64
        const uint64_t fc = A * (uint64_t)k.nc;
        b.c[d] = ci;
        b.s[d] = (int)__umul64hi(fc, (uint64_t)kSub);
        b.fc[d] = fc;
        // window anchor (Sec. 2.2): a = floor(y/h + (P odd)/2) - ceil(P/2) + 1,
        // the P support points are a + l, l = 0..P-1
        uint64_t gi = __umul64hi(A, (uint64_t)k.M), fg = A * (uint64_t)k.M;
        if (k.odd_P) {
            const uint64_t f2 = fg + (1ull << 63);
            gi += f2 < fg ? 1ull : 0ull;
            fg = f2;
        }
        b.fg[d] = fg;
        int ai = ((int)gi - k.ceilP2 + 1) % k.M;
        if (ai < 0)
            ai += k.M;
        b.a[d] = ai;
        b.tl[d] = ai / k.T;
    }
    return b;
}

__device__ __forceinline__ void bin_keys_body(const KeyArgs &k, int64_t i)
{
    if (i >= k.N)
        return;
    Bin b = compute_bin(k, i);
    if (b.bad)
        atomicOr(k.err, 1);
    int kn = ((b.c[2] * k.nc + b.c[1]) * k.nc + b.c[0]) * kSub3 +
             (b.s[2] * kSub + b.s[1]) * kSub + b.s[0];
    int kt = (b.tl[2] * k.nt + b.tl[1]) * k.nt + b.tl[0];
    k.keyn[i] = kn;
    k.keyt[i] = kt;
    k.slotn[i] = atomicAdd(&k.cntn[kn], 1);
    k.slott[i] = atomicAdd(&k.cntt[kt], 1);
}

// a fraction held as a 64-bit word (times 2^64) in [0, 1]: its top 32 bits
// (FP32), or 53 bits (FP64)
template <typename R>
__device__ __forceinline__ R frac64(uint64_t f);
template <>
__device__ __forceinline__ float frac64<float>(uint64_t f)
{
    return __uint2float_rn((unsigned)(f >> 32)) * 2.3283064365386963e-10f;
}
template <>
__device__ __forceinline__ double frac64<double>(uint64_t f)
{
    return __ull2double_rn(f >> 11) * 1.1102230246251565e-16;
}

template <typename R, typename R4>
__device__ __forceinline__ void bin_scatter_body(const KeyArgs &k, int64_t i)
{
    if (i >= k.N)
        return;
    Bin b = compute_bin(k, i);
    int pn = k.startn[k.keyn[i]] + k.slotn[i];
    int pt = k.startt[k.keyt[i]] + k.slott[i];
    R4 *tdat = (R4 *)k.tdat, *tfrc = (R4 *)k.tfrc;
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;  // set_positions: forces come later
    if (k.f) {
        f0 = k.f[3 * i];
        f1 = k.f[3 * i + 1];
        f2 = k.f[3 * i + 2];
    }
    if (k.nrec) {
        // FP32 near record (32 bytes): cell-local position in cell units split
        // hi + lo, hi on a 2^-20 lattice stored as three 21-bit integers
        // (exact in FP32 together with an integer colleague offset, so hi
        // differences are exact), |lo| <= 2^-21 (FP32: 2^-45 absolute), and
        // the force:
        //   (lo.x, lo.y, lo.z, f.x) (f.y, f.z, bits 0..31, bits 32..63 of
        //   hi.x | hi.y << 21 | hi.z << 42)
        float lo[3];
        uint64_t hq[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // hi = the fraction rounded to 20 bits (0 .. 2^20), lo = the rest
            // (|lo| <= 2^43 units of 2^-64, exact as a signed word; the word
            // wraps when hi = 2^20), converted from two exact halves
            const uint64_t fc = b.fc[d];
            hq[d] = (fc >> 44) + ((fc >> 43) & 1ull);
            const long long lw = (long long)(fc - (hq[d] << 44));
            lo[d] = fmaf((float)(int)(lw >> 21), 2097152.f, (float)(int)(lw & 0x1FFFFFll)) * 5.421010862427522e-20f;
        }
        const uint64_t packed = hq[0] | (hq[1] << 21) | (hq[2] << 42);
        const float fx = (float)f0, fy = (float)f1, fz = (float)f2;
        float4 *rec = (float4 *)k.nrec + 2 * (int64_t)pn;
        rec[0] = make_float4(lo[0], lo[1], lo[2], fx);
        rec[1] = make_float4(fy, fz, __uint_as_float((unsigned)packed), __uint_as_float((unsigned)(packed >> 32)));
        if (k.nflo) {  // double-single P2P: the forces' FP32 rounding errors
            float4 fl = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k.f)
                fl = make_float4((float)(f0 - (double)fx), (float)(f1 - (double)fy), (float)(f2 - (double)fz), 0.f);
            ((float4 *)k.nflo)[pn] = fl;
        }
    } else {
        R4 pos;
        pos.x = (R)(__ull2double_rn(b.fc[0]) * 5.421010862427522e-20 * k.cell);
        pos.y = (R)(__ull2double_rn(b.fc[1]) * 5.421010862427522e-20 * k.cell);
        pos.z = (R)(__ull2double_rn(b.fc[2]) * 5.421010862427522e-20 * k.cell);
        pos.w = (R)0;
        ((R4 *)k.npos)[pn] = pos;
    }
    k.permn[pn] = (int32_t)i;
    int packed = (b.a[0] - b.tl[0] * k.T) | ((b.a[1] - b.tl[1] * k.T) << 4) |
                 ((b.a[2] - b.tl[2] * k.T) << 8);
    R4 td;
    td.x = frac64<R>(b.fg[0]);
    td.y = frac64<R>(b.fg[1]);
    td.z = frac64<R>(b.fg[2]);
    td.w = (R)packed;  // small integer, exact in FP32 and FP64
    tdat[pt] = td;
    k.permt[pt] = (int32_t)i;
    if (k.f) {
        R4 fv;
        fv.x = (R)f0;
        fv.y = (R)f1;
        fv.z = (R)f2;
        fv.w = (R)0;
        if (!k.nrec)
            ((R4 *)k.nfrc)[pn] = fv;
        if (k.tf_ds)
            store_force_ds((float4 *)k.tfrc + 2 * (int64_t)pt, f0, f1, f2);
        else
            tfrc[pt] = fv;
    }
}

// Forces into both sorted orders: FP64 near forces as 4-vectors (nfrc), or
// into the force slots of the FP32 near records (floats 3, 4, 5 of each 8)
// with their FP32 rounding errors in nflo for the double-single P2P.
template <typename R, typename R4>
__global__ void k_gather_forces(const double *__restrict__ f, const int32_t *__restrict__ permn,
                                const int32_t *__restrict__ permt, dvec4 *nfrc, float *nrec,
                                float4 *nflo, R4 *tfrc, bool tf_ds, int64_t N)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N)
        return;
    int in = permn[p], it = permt[p];
    if (nrec) {
        float *r = nrec + 8 * p;
        const float fx = (float)f[3 * in], fy = (float)f[3 * in + 1], fz = (float)f[3 * in + 2];
        r[3] = fx;
        r[4] = fy;
        r[5] = fz;
        if (nflo)
            nflo[p] = make_float4((float)(f[3 * in] - (double)fx), (float)(f[3 * in + 1] - (double)fy),
                                  (float)(f[3 * in + 2] - (double)fz), 0.f);
    } else {
        dvec4 a;
        a.x = f[3 * in];
        a.y = f[3 * in + 1];
        a.z = f[3 * in + 2];
        a.w = 0.0;
        nfrc[p] = a;
    }
    if (tf_ds) {
        store_force_ds((float4 *)tfrc + 2 * p, f[3 * it], f[3 * it + 1], f[3 * it + 2]);
        return;
    }
    R4 b;
    b.x = (R)f[3 * it];
    b.y = (R)f[3 * it + 1];
    b.z = (R)f[3 * it + 2];
    b.w = (R)0;
    tfrc[p] = b;
}

// Exclusive scans of up to three count arrays, one block each (blockIdx.x
// picks the job); out[n] receives the total.  With `chunk` > 0 the values
// scanned are the P2P work items of each cell group (p2p_group_cell),
// ceil(count / chunk) with count the sum of its sub-cell counts `in`, instead
// of in[i].
struct ScanJob {
    const int32_t *in;
    int32_t *out;
    int n, chunk, nc, K;
};

__device__ __forceinline__ int scan_value(const ScanJob &j, int i)
{
    if (j.chunk <= 0)
        return j.in[i];
    int ncg;
    const int c = p2p_group_cell(i, j.nc, j.K, ncg);
    int cnt = 0;
    for (int k = 0; k < ncg * kSub3; ++k)
        cnt += j.in[c * kSub3 + k];
    return (cnt + j.chunk - 1) / j.chunk;
}

__device__ __forceinline__ void scan_body(const ScanJob &j)
{
    __shared__ int32_t wsum[32];
    const int n = j.n;
    int32_t *__restrict__ out = j.out;
    int tid = threadIdx.x, nthr = blockDim.x;
    int per = (n + nthr - 1) / nthr;
    int lo = min(tid * per, n), hi = min(lo + per, n);
    int s = 0;
    for (int i = lo; i < hi; ++i)
        s += scan_value(j, i);
    int lane = tid & 31, w = tid >> 5;
    int v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    if (lane == 31)
        wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = nthr >> 5;
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += u;
        }
        if (lane < nw)
            wsum[lane] = t;  // inclusive prefix of warp totals
    }
    __syncthreads();
    int run = v - s + (w > 0 ? wsum[w - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        int c = scan_value(j, i);
        out[i] = run;
        run += c;
    }
    if (tid == nthr - 1)
        out[n] = run;
}

__global__ void k_bin_keys(KeyArgs k)
{
    bin_keys_body(k, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}
// One plan's scatter, which also zeroes the per-key and per-tile counters
// for the next binning: the scans have consumed them (the keys kernel of the
// next binning counts into them again).
template <typename R, typename R4>
__global__ void k_bin_scatter(KeyArgs k)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    bin_scatter_body<R, R4>(k, i);
    for (int64_t q = i; q < k.ncntn; q += stride)
        k.cntn[q] = 0;
    for (int64_t q = i; q < k.ncntt; q += stride)
        k.cntt[q] = 0;
}
__global__ void __launch_bounds__(1024) k_scan(ScanJob j0, ScanJob j1, ScanJob j2)
{
    scan_body(blockIdx.x == 0 ? j0 : (blockIdx.x == 1 ? j1 : j2));
}

// Many plans' boxes in one launch: a block finds its box by binary search over
// the boxes' block offsets (base) and runs the same body on that box's data.
__global__ void k_bin_keys_boxes(const KeyArgs *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    bin_keys_body(boxes[b], (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x);
}
template <typename R, typename R4>
__global__ void k_bin_scatter_boxes(const KeyArgs *__restrict__ boxes, const int *__restrict__ base, int nbox)
{
    const int b = find_box(base, nbox, (int)blockIdx.x);
    bin_scatter_body<R, R4>(boxes[b], (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x);
}
__global__ void __launch_bounds__(1024) k_scan_jobs(const ScanJob *__restrict__ jobs)
{
    scan_body(jobs[blockIdx.x]);
}
// zero n[k] int32 values at p[k] for every job k (threads over the
// concatenated ranges, base = prefix offsets in blocks of 256)
struct ZeroJob {
    int32_t *p;
    int n;
};
__global__ void k_zero_jobs(const ZeroJob *__restrict__ jobs, const int *__restrict__ base, int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const int i = ((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x;
    if (i < jobs[b].n)
        jobs[b].p[i] = 0;
}

// Step a7 (Algorithm 1, SUM): u = u^N + u^F in FP64, user order (the self
// term is already in u^N, see k_p2p.cu).
template <typename R>
__global__ void k_sum(const R *__restrict__ un, const R *__restrict__ uf, double *__restrict__ u,
                      int64_t n3)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3)
        return;
    u[i] = (double)un[i] + (double)uf[i];
}

// elementwise jobs of many boxes: the sum (src = u^N, src2 = u^F), or a copy
// with conversion (src2 unused)
struct EltJob {
    const void *src, *src2;
    void *dst;
    int64_t n;
};
template <typename R>
__global__ void k_sum_jobs(const EltJob *__restrict__ jobs, const int *__restrict__ base, int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const EltJob &j = jobs[b];
    const int64_t i = (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x;
    if (i < j.n)
        ((double *)j.dst)[i] = (double)((const R *)j.src)[i] + (double)((const R *)j.src2)[i];
}
template <typename A, typename B>
__global__ void k_convert_jobs(const EltJob *__restrict__ jobs, const int *__restrict__ base, int njob)
{
    const int b = find_box(base, njob, (int)blockIdx.x);
    const EltJob &j = jobs[b];
    const int64_t i = (int64_t)((int)blockIdx.x - base[b]) * blockDim.x + threadIdx.x;
    if (i < j.n)
        ((B *)j.dst)[i] = (B)((const A *)j.src)[i];
}

template <typename R>
__global__ void k_copy_out(const R *__restrict__ src, double *__restrict__ dst, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        dst[i] = (double)src[i];
}

template <typename A, typename B>
__global__ void k_convert(const A *__restrict__ src, B *__restrict__ dst, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        dst[i] = (B)src[i];
}

KeyArgs key_args(ewald_plan_s *p, const BinArgs &a)
{
    KeyArgs k;
    k.x = a.x;
    k.f = a.f;
    k.N = a.N;
    k.L = a.L;
    k.inv_L = 1.0 / a.L;
    k.cell = a.cell;
    k.fix_scale = 4611686018427387904.0 / a.L;  // 2^62 / L
    std::memcpy(&k.L_bits, &a.L, sizeof(double));
    k.odd_P = a.P % 2;
    k.nc = a.nc;
    k.M = a.M;
    k.T = a.T;
    k.nt = a.nt;
    k.ceilP2 = (a.P + 1) / 2;
    k.keyn = p->keyn;
    k.slotn = p->slotn;
    k.keyt = p->keyt;
    k.slott = p->slott;
    k.cntn = p->cntn;
    k.cntt = p->cntt;
    k.ncntn = p->g.nkeys;
    k.ncntt = p->g.ntiles;
    k.permn = p->permn;
    k.permt = p->permt;
    k.startn = p->startn;
    k.startt = p->startt;
    k.npos = p->npos;
    k.nfrc = p->nfrc;
    k.nrec = p->nrec;
    k.nflo = p->nflo;
    k.tdat = p->tdat;
    k.tfrc = p->tfrc;
    k.tf_ds = a.tf_ds;
    k.err = p->err;
    return k;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_bin_keys(ewald_plan_s *p, const BinArgs &a, cudaStream_t s)
{
    KeyArgs k = key_args(p, a);
    k_bin_keys<<<blocks_for(a.N, 256), 256, 0, s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *in, int32_t *out, int n, cudaStream_t s)
{
    ScanJob j{in, out, n, 0, 0, 0};
    k_scan<<<1, 1024, 0, s>>>(j, j, j);
    return cudaGetLastError();
}

cudaError_t launch_bin_scans(ewald_plan_s *p, cudaStream_t s)
{
    const Geometry &g = p->g;
    k_scan<<<3, 1024, 0, s>>>(ScanJob{p->cntn, p->startn, g.nkeys, 0, 0, 0},
                              ScanJob{p->cntt, p->startt, g.ntiles, 0, 0, 0},
                              ScanJob{p->cntn, p->item_off, p2p_groups(g.nc, g.K), kP2PChunk, g.nc, g.K});
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(ewald_plan_s *p, const BinArgs &a, cudaStream_t s)
{
    KeyArgs k = key_args(p, a);
    if (a.f64)
        k_bin_scatter<double, dvec4><<<blocks_for(a.N, 256), 256, 0, s>>>(k);
    else
        k_bin_scatter<float, float4><<<blocks_for(a.N, 256), 256, 0, s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_gather_forces(ewald_plan_s *p, const double *f, cudaStream_t s)
{
    if (p->near64)
        k_gather_forces<double, dvec4><<<blocks_for(p->N, 256), 256, 0, s>>>(
            f, p->permn, p->permt, (dvec4 *)p->nfrc, (float *)p->nrec, (float4 *)p->nflo,
            (dvec4 *)p->tfrc, p->grid_ds, p->N);
    else
        k_gather_forces<float, float4><<<blocks_for(p->N, 256), 256, 0, s>>>(
            f, p->permn, p->permt, nullptr, (float *)p->nrec, nullptr, (float4 *)p->tfrc, false, p->N);
    return cudaGetLastError();
}

// P2P work items per cell (chunks of at most kP2PChunk targets) and their
// prefix offsets, in one launch.
cudaError_t launch_cell_items(ewald_plan_s *p, cudaStream_t s)
{
    ScanJob j{p->cntn, p->item_off, p2p_groups(p->g.nc, p->g.K), kP2PChunk, p->g.nc, p->g.K};
    k_scan<<<1, 1024, 0, s>>>(j, j, j);
    return cudaGetLastError();
}

cudaError_t launch_sum(ewald_plan_s *p, const double *f, double *u, cudaStream_t s)
{
    (void)f;
    int64_t n3 = 3 * p->N;
    if (p->near64)
        k_sum<double><<<blocks_for(n3, 256), 256, 0, s>>>((const double *)p->un,
                                                          (const double *)p->uf, u, n3);
    else
        k_sum<float><<<blocks_for(n3, 256), 256, 0, s>>>((const float *)p->un,
                                                         (const float *)p->uf, u, n3);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const void *src, bool src_f64, double *dst, int64_t n, cudaStream_t s)
{
    if (src_f64)
        k_copy_out<double><<<blocks_for(n, 256), 256, 0, s>>>((const double *)src, dst, n);
    else
        k_copy_out<float><<<blocks_for(n, 256), 256, 0, s>>>((const float *)src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_grid_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t n,
                                cudaStream_t s)
{
    unsigned nb = blocks_for(n, 256);
    if (src_f64 && dst_f64)
        k_convert<double, double><<<nb, 256, 0, s>>>((const double *)src, (double *)dst, n);
    else if (src_f64)
        k_convert<double, float><<<nb, 256, 0, s>>>((const double *)src, (float *)dst, n);
    else if (dst_f64)
        k_convert<float, double><<<nb, 256, 0, s>>>((const float *)src, (double *)dst, n);
    else
        k_convert<float, float><<<nb, 256, 0, s>>>((const float *)src, (float *)dst, n);
    return cudaGetLastError();
}

// ---- many plans' binning and sums in one launch per kernel (batches) -------
namespace {
template <typename T>
cudaError_t upload(const std::vector<T> &v, T **d)
{
    *d = nullptr;
    if (v.empty())
        return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)d, sizeof(T) * v.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}
// prefix offsets (in blocks of 256) over per-box element counts
std::vector<int> block_base(const std::vector<int64_t> &n, unsigned &grid)
{
    std::vector<int> b(1, 0);
    for (int64_t v : n)
        b.push_back(b.back() + (int)((v + 255) / 256));
    grid = (unsigned)b.back();
    return b;
}
}  // namespace

struct BinBoxes {
    KeyArgs *keys = nullptr, *scat[2] = {nullptr, nullptr};  // scat[0]: FP32 records, [1]: FP64
    int *keys_base = nullptr, *scat_base[2] = {nullptr, nullptr}, *zero_base = nullptr;
    int nkeys = 0, nscat[2] = {0, 0}, nzero = 0, njobs = 0;
    unsigned keys_grid = 0, scat_grid[2] = {0, 0}, zero_grid = 0;
    ScanJob *jobs = nullptr;
    ZeroJob *zero = nullptr;
    // sums (u = u^N + u^F), by result precision: [0] FP32, [1] FP64
    EltJob *sum[2] = {nullptr, nullptr};
    int *sum_base[2] = {nullptr, nullptr}, nsum[2] = {0, 0};
    unsigned sum_grid[2] = {0, 0};
};

cudaError_t bin_boxes_create(ewald_plan_s *const *plans, const double *const *x, const double *const *f,
                             double *const *u, int n, BinBoxes **out)
{
    BinBoxes *b = new (std::nothrow) BinBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    std::vector<KeyArgs> keys, scat[2];
    std::vector<int64_t> nk, ns[2], nz, nsum[2];
    std::vector<ScanJob> jobs;
    std::vector<ZeroJob> zero;
    std::vector<EltJob> sum[2];
    for (int i = 0; i < n; ++i) {
        ewald_plan_s *p = plans[i];
        const Geometry &g = p->g;
        BinArgs a;
        a.x = x[i];
        a.f = f[i];
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
        const KeyArgs k = key_args(p, a);
        keys.push_back(k);
        nk.push_back(p->N);
        scat[a.f64 ? 1 : 0].push_back(k);
        ns[a.f64 ? 1 : 0].push_back(p->N);
        jobs.push_back(ScanJob{p->cntn, p->startn, g.nkeys, 0, 0, 0});
        jobs.push_back(ScanJob{p->cntt, p->startt, g.ntiles, 0, 0, 0});
        jobs.push_back(ScanJob{p->cntn, p->item_off, p2p_groups(g.nc, g.K), kP2PChunk, g.nc, g.K});
        zero.push_back(ZeroJob{p->cntn, g.nkeys});
        nz.push_back(g.nkeys);
        zero.push_back(ZeroJob{p->cntt, g.ntiles});
        nz.push_back(g.ntiles);
        const int r = p->near64 ? 1 : 0;
        sum[r].push_back(EltJob{p->un, p->uf, u[i], 3 * p->N});
        nsum[r].push_back(3 * p->N);
        p->positions_valid = true;
    }
    cudaError_t e = cudaSuccess;
    std::vector<int> kb = block_base(nk, b->keys_grid), zb = block_base(nz, b->zero_grid);
    b->nkeys = (int)keys.size();
    b->nzero = (int)zero.size();
    b->njobs = (int)jobs.size();
    if (e == cudaSuccess) e = upload(keys, &b->keys);
    if (e == cudaSuccess) e = upload(kb, &b->keys_base);
    if (e == cudaSuccess) e = upload(jobs, &b->jobs);
    if (e == cudaSuccess) e = upload(zero, &b->zero);
    if (e == cudaSuccess) e = upload(zb, &b->zero_base);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        std::vector<int> sb = block_base(ns[r], b->scat_grid[r]), ub = block_base(nsum[r], b->sum_grid[r]);
        b->nscat[r] = (int)scat[r].size();
        b->nsum[r] = (int)sum[r].size();
        e = upload(scat[r], &b->scat[r]);
        if (e == cudaSuccess) e = upload(sb, &b->scat_base[r]);
        if (e == cudaSuccess) e = upload(sum[r], &b->sum[r]);
        if (e == cudaSuccess) e = upload(ub, &b->sum_base[r]);
    }
    if (e != cudaSuccess) {
        bin_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

// counters zeroed, keys, the three scans per box, scatter: every box's
// binning in four launches (five with both record precisions)
cudaError_t bin_boxes_launch(const BinBoxes *b, cudaStream_t s)
{
    if (b->nzero)
        k_zero_jobs<<<b->zero_grid, 256, 0, s>>>(b->zero, b->zero_base, b->nzero);
    if (b->nkeys)
        k_bin_keys_boxes<<<b->keys_grid, 256, 0, s>>>(b->keys, b->keys_base, b->nkeys);
    if (b->njobs)
        k_scan_jobs<<<b->njobs, 1024, 0, s>>>(b->jobs);
    if (b->nscat[0])
        k_bin_scatter_boxes<float, float4><<<b->scat_grid[0], 256, 0, s>>>(b->scat[0], b->scat_base[0], b->nscat[0]);
    if (b->nscat[1])
        k_bin_scatter_boxes<double, dvec4><<<b->scat_grid[1], 256, 0, s>>>(b->scat[1], b->scat_base[1], b->nscat[1]);
    return cudaGetLastError();
}

cudaError_t sum_boxes_launch(const BinBoxes *b, cudaStream_t s)
{
    if (b->nsum[0])
        k_sum_jobs<float><<<b->sum_grid[0], 256, 0, s>>>(b->sum[0], b->sum_base[0], b->nsum[0]);
    if (b->nsum[1])
        k_sum_jobs<double><<<b->sum_grid[1], 256, 0, s>>>(b->sum[1], b->sum_base[1], b->nsum[1]);
    return cudaGetLastError();
}

int bin_boxes_launches(const BinBoxes *b)
{
    return (b->nzero ? 1 : 0) + (b->nkeys ? 1 : 0) + (b->njobs ? 1 : 0) + (b->nscat[0] ? 1 : 0) +
           (b->nscat[1] ? 1 : 0);
}
int sum_boxes_launches(const BinBoxes *b) { return (b->nsum[0] ? 1 : 0) + (b->nsum[1] ? 1 : 0); }

void bin_boxes_destroy(BinBoxes *b)
{
    if (!b)
        return;
    void *ptrs[] = {b->keys, b->scat[0], b->scat[1], b->keys_base, b->scat_base[0], b->scat_base[1], b->zero_base,
                    b->jobs, b->zero, b->sum[0], b->sum[1], b->sum_base[0], b->sum_base[1]};
    for (void *q : ptrs)
        if (q)
            cudaFree(q);
    delete b;
}

// FP64 grids -> FP32 copies for G2P, many boxes (jobs: src FP64, dst FP32, n)
struct ConvBoxes {
    EltJob *jobs = nullptr;
    int *base = nullptr, n = 0;
    unsigned grid = 0;
};
cudaError_t conv_boxes_create(const std::vector<const void *> &src, const std::vector<void *> &dst,
                              const std::vector<int64_t> &n, ConvBoxes **out)
{
    ConvBoxes *b = new (std::nothrow) ConvBoxes;
    if (!b)
        return cudaErrorMemoryAllocation;
    std::vector<EltJob> jobs;
    for (size_t i = 0; i < src.size(); ++i)
        jobs.push_back(EltJob{src[i], nullptr, dst[i], n[i]});
    std::vector<int> base = block_base(n, b->grid);
    b->n = (int)jobs.size();
    cudaError_t e = upload(jobs, &b->jobs);
    if (e == cudaSuccess)
        e = upload(base, &b->base);
    if (e != cudaSuccess) {
        conv_boxes_destroy(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}
cudaError_t conv_boxes_launch(const ConvBoxes *b, cudaStream_t s)
{
    if (b->n)
        k_convert_jobs<double, float><<<b->grid, 256, 0, s>>>(b->jobs, b->base, b->n);
    return cudaGetLastError();
}
int conv_boxes_launches(const ConvBoxes *b) { return b && b->n ? 1 : 0; }

void conv_boxes_destroy(ConvBoxes *b)
{
    if (!b)
        return;
    if (b->jobs)
        cudaFree(b->jobs);
    if (b->base)
        cudaFree(b->base);
    delete b;
}

}  // namespace ewg
