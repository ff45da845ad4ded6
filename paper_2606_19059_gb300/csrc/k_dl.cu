// k_dl.cu -- the double-layer (stresslet) part of the combined single and
// double layer potential of Sec. 2.3: every source carries two vectors q and
// n, and the sum over sources and images of T(x_i - y_j + p) applied to
// q_j (x) n_j is added to the Stokeslet sum.
//
// The paper leaves T and its split T = T^N + T^F to another work.  Here
// T_jlm(r) = -6 r_j r_l r_m / r^5 (the stresslet of the Stokeslet
// I/r + r r^T/r^3), and the split screens T = 2 [d_m G_jl - delta_jl d_m phi
// + delta_jm d_l phi + delta_lm d_j phi] (phi = 1/r) the way eq. (g-near)
// screens G:
//   T^N(r) : D = 2 beta r (r.D.r) + 2 gamma (r tr D + (D + D^T) r),
//     beta  = -3 erfc(xi r)/r^5 - (2 xi/sqrt(pi)) (3/r^4 + 2 xi^2/r^2) e^{-xi^2 r^2},
//     gamma = (2 xi^3/sqrt(pi)) e^{-xi^2 r^2};
//   T-hat^F(k) : D-hat = 8 pi i H(k) [(D-hat + D-hat^T) k + k tr D-hat
//                         - 2 k (k.D-hat.k)/k^2] / k^2,
//     H(k) = (1 + k^2/(4 xi^2)) e^{-k^2/(4 xi^2)} (the Stokeslet's screening).
// Only the symmetric part S of D = q (x) n enters, so the far field spreads
// six components (S_xx, S_yy, S_zz) and (S_xy, S_xz, S_yz) -- two triples
// through the Stokeslet's own P2G kernel and batched FFT -- where the paper
// spreads nine; the CNV adds the double layer's v-hat into the Stokeslet's
// before the one inverse FFT and G2P.  T^F is odd: no self term.
//
// Kernels: k_dl_densities (tile-order S, the P2G input format), k_scale_dl
// (CNV, HBM-bound: 6 complex components in, 3 read-modify-written), and the
// near field in two forms.  FP32 plans: k_dl_records (48-byte near-order
// records: the Stokeslet records' cell-local position parts and S in FP32)
// for k_p2p_dl32 in k_p2p.cu, the Stokeslet P2P machinery with the
// double-layer pair.  Plans with FP64 FFTs or kernels: k_dl_sort (near-sorted
// copies of positions, q and n) and k_p2p_dl (an FP32 distance filter over the
// (2K+1)^3 neighbour cells of the plan's cell lists, then FP64 pair arithmetic
// for queued in-range pairs only, summed in FP64).
#include "internal.h"

namespace ewg {
namespace {

template <typename R4>
__global__ void __launch_bounds__(256) k_dl_densities(const double *__restrict__ q, const double *__restrict__ n,
                                                      const int32_t *__restrict__ permt, int64_t N,
                                                      R4 *__restrict__ sd, R4 *__restrict__ so, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N)
        return;
    const int64_t i = permt[t];
    const double q0 = q[3 * i], q1 = q[3 * i + 1], q2 = q[3 * i + 2];
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    if (!(isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(n0) && isfinite(n1) && isfinite(n2)))
        atomicOr(err, 1);
    R4 a, b;
    a.x = q0 * n0;
    a.y = q1 * n1;
    a.z = q2 * n2;
    a.w = 0;
    b.x = 0.5 * (q0 * n1 + q1 * n0);
    b.y = 0.5 * (q0 * n2 + q2 * n0);
    b.z = 0.5 * (q1 * n2 + q2 * n1);
    b.w = 0;
    sd[t] = a;
    so[t] = b;
}

// The same densities for double-single grid kernels: per point and triple the
// FP32 high parts and their rounding errors, (h.xyz, 0), (l.xyz, 0).
__global__ void __launch_bounds__(256) k_dl_densities_ds(const double *__restrict__ q, const double *__restrict__ n,
                                                         const int32_t *__restrict__ permt, int64_t N,
                                                         float4 *__restrict__ sd, float4 *__restrict__ so, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N)
        return;
    const int64_t i = permt[t];
    const double q0 = q[3 * i], q1 = q[3 * i + 1], q2 = q[3 * i + 2];
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    if (!(isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(n0) && isfinite(n1) && isfinite(n2)))
        atomicOr(err, 1);
    const double a[3] = {q0 * n0, q1 * n1, q2 * n2};
    const double b[3] = {0.5 * (q0 * n1 + q1 * n0), 0.5 * (q0 * n2 + q2 * n0), 0.5 * (q1 * n2 + q2 * n1)};
    float ah[3], bh[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ah[k] = (float)a[k];
        bh[k] = (float)b[k];
    }
    sd[2 * t] = make_float4(ah[0], ah[1], ah[2], 0.f);
    sd[2 * t + 1] = make_float4((float)(a[0] - (double)ah[0]), (float)(a[1] - (double)ah[1]),
                                (float)(a[2] - (double)ah[2]), 0.f);
    so[2 * t] = make_float4(bh[0], bh[1], bh[2], 0.f);
    so[2 * t + 1] = make_float4((float)(b[0] - (double)bh[0]), (float)(b[1] - (double)bh[1]),
                                (float)(b[2] - (double)bh[2]), 0.f);
}

template <typename R, typename C2>
__device__ __forceinline__ C2 cmad(C2 a, R k, C2 acc)
{
    acc.x = fma(a.x, k, acc.x);
    acc.y = fma(a.y, k, acc.y);
    return acc;
}

// v-hat += C t(kx) t(ky) t(kz) (1 + k^2/(4 xi^2)) / k^2 * i [2 S k + k (tr S - 2 k.S.k / k^2)]
// with t the plan's CNV table (e^{-k^2/(4 xi^2)} / w-hat^2 per axis, 0 on the
// Nyquist plane) and C = 8 pi h^3 / M^3, as the Stokeslet's CNV.
template <typename R, typename C2>
__global__ void __launch_bounds__(256) k_scale_dl(C2 *__restrict__ spec, const C2 *__restrict__ sa,
                                                  const C2 *__restrict__ sb, const R *__restrict__ tab, int M,
                                                  int Mh, int64_t ncplx, R kfac, R inv4xi2, R C)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncplx)
        return;
    const int ix = (int)(idx % Mh);
    const int iy = (int)((idx / Mh) % M);
    const int iz = (int)(idx / ((int64_t)Mh * M));
    const int ny = iy <= M / 2 ? iy : iy - M;
    const int nz = iz <= M / 2 ? iz : iz - M;
    const R kx = kfac * ix, ky = kfac * ny, kz = kfac * nz;
    const R k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 > (R)0))
        return;  // the k = 0 mode stays dropped
    const R s = C * tab[ix] * tab[iy] * tab[iz] * ((R)1 + k2 * inv4xi2) / k2;
    const C2 Sxx = sa[idx], Syy = sa[ncplx + idx], Szz = sa[2 * ncplx + idx];
    const C2 Sxy = sb[idx], Sxz = sb[ncplx + idx], Syz = sb[2 * ncplx + idx];
    C2 z;
    z.x = (R)0;
    z.y = (R)0;
    // S k
    const C2 ax = cmad<R>(Sxz, kz, cmad<R>(Sxy, ky, cmad<R>(Sxx, kx, z)));
    const C2 ay = cmad<R>(Syz, kz, cmad<R>(Syy, ky, cmad<R>(Sxy, kx, z)));
    const C2 az = cmad<R>(Szz, kz, cmad<R>(Syz, ky, cmad<R>(Sxz, kx, z)));
    // c = tr S - 2 k.S.k / k^2
    const C2 kSk = cmad<R>(az, kz, cmad<R>(ay, ky, cmad<R>(ax, kx, z)));
    const R m2 = (R)-2 / k2;
    C2 c;
    c.x = fma(kSk.x, m2, Sxx.x + Syy.x + Szz.x);
    c.y = fma(kSk.y, m2, Sxx.y + Syy.y + Szz.y);
    const C2 a[3] = {ax, ay, az};
    const R kk[3] = {kx, ky, kz};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // w = 2 (S k)_j + k_j c; v = i s w
        const R wx = fma(kk[j], c.x, (R)2 * a[j].x), wy = fma(kk[j], c.y, (R)2 * a[j].y);
        C2 v = spec[j * ncplx + idx];
        v.x = fma(-s, wy, v.x);
        v.y = fma(s, wx, v.y);
        spec[j * ncplx + idx] = v;
    }
}

struct DlNearArgs {
    const int32_t *permn, *keyn, *startn;
    const dvec4 *pos, *qs, *ns;       // near-sorted: wrapped positions, q, n (FP64 pairs)
    const float4 *lhi, *llo;          // near-sorted cell-local positions in cell units, hi + lo parts
    const float4 *q32, *n32;          // near-sorted q, n in FP32 (FP32 pairs)
    double *u;
    int64_t N;
    double L, xi, rc2;
    float w;                          // cell width
    float rcm2;                       // FP32 filter threshold, cell units: rc / w grown past the lo parts
    int nc, K;
};

// near-sorted copies (slot s holds source permn[s]): wrapped positions, q and
// n in FP64; the cell-local position in cell units, q = x / cell - c, as FP32
// parts hi (rounded to a 2^-20 lattice, so hi minus an integer neighbour
// offset and differences of such values are exact in FP32) and lo = q - hi
// (|lo| <= 2^-21); q and n in FP32
__global__ void __launch_bounds__(256) k_dl_sort(const double *__restrict__ x, const double *__restrict__ q,
                                                 const double *__restrict__ n, const int32_t *__restrict__ permn,
                                                 const int32_t *__restrict__ keyn, int64_t N, double L,
                                                 double inv_L, double inv_cell, int nc, dvec4 *pos, dvec4 *qs,
                                                 dvec4 *ns, float4 *lhi, float4 *llo, float4 *q32, float4 *n32)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N)
        return;
    const int64_t j = permn[s];
    const int c = keyn[j] / kSub3;
    const int cc[3] = {c % nc, (c / nc) % nc, c / (nc * nc)};
    double w[3];
    float h[3], l[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        w[d] = wrap_coord(x[3 * j + d], L, inv_L);
        const double qd = w[d] * inv_cell - cc[d];
        const double X = rint(qd * 1048576.0) * (1.0 / 1048576.0);
        h[d] = (float)X;
        l[d] = (float)(qd - X);
    }
    dvec4 v;
    v.x = w[0];
    v.y = w[1];
    v.z = w[2];
    v.w = 0.0;
    pos[s] = v;
    lhi[s] = make_float4(h[0], h[1], h[2], 0.f);
    llo[s] = make_float4(l[0], l[1], l[2], 0.f);
    dvec4 a, b;
    a.x = q[3 * j];
    a.y = q[3 * j + 1];
    a.z = q[3 * j + 2];
    a.w = 0.0;
    b.x = n[3 * j];
    b.y = n[3 * j + 1];
    b.z = n[3 * j + 2];
    b.w = 0.0;
    qs[s] = a;
    ns[s] = b;
    q32[s] = make_float4((float)a.x, (float)a.y, (float)a.z, 0.f);
    n32[s] = make_float4((float)b.x, (float)b.y, (float)b.z, 0.f);
}

__device__ __forceinline__ int floor_div(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

constexpr int kDlWarps = 4;
constexpr int kDlQ = 16;  // queued in-range sources per lane before an evaluation round

struct DlQueue {
    int src[kDlQ][32];   // [entry][lane]: a lane touches only its own column
    int code[kDlQ][32];  // neighbour cell offset (ox, oy, oz), each biased by 64 into 8 bits
};

// T^N(r) : S of one pair, r = target - source image, in precision R
template <typename R>
__device__ __forceinline__ void dl_pair(R r0, R r1, R r2, R rr2, R q0, R q1, R q2, R n0, R n1, R n2, R xi,
                                        R c_e, R &u0, R &u1, R &u2)
{
    const R qr = fma(q0, r0, fma(q1, r1, q2 * r2));
    const R nr = fma(n0, r0, fma(n1, r1, n2 * r2));
    const R qn = fma(q0, n0, fma(q1, n1, q2 * n2));
    const R rr = sqrt(rr2), inv2 = (R)1 / rr2;
    const R e = exp(-xi * xi * rr2);
    const R beta = (R)-3 * erfc(xi * rr) * inv2 * inv2 / rr - c_e * ((R)3 * inv2 * inv2 + (R)2 * xi * xi * inv2) * e;
    const R gamma = c_e * xi * xi * e;
    // 2 beta r (q.r)(n.r) + 2 gamma (r q.n + q n.r + n q.r)
    const R br = (R)2 * beta * qr * nr, g2 = (R)2 * gamma;
    u0 += br * r0 + g2 * (r0 * qn + q0 * nr + n0 * qr);
    u1 += br * r1 + g2 * (r1 * qn + q1 * nr + n1 * qr);
    u2 += br * r2 + g2 * (r2 * qn + q2 * nr + n2 * qr);
}

// u_i += sum over sources j and images within rc of T^N(x_i - y_j - p) : S_j.
// One warp per 32 near-sorted targets, one lane per target.  Each lane walks
// the sources of its (2K+1)^3 neighbour cells with an FP32 distance test on
// cell-local coordinates (threshold rc grown past FP32 rounding) and queues
// the sources that pass; when a lane's queue is full, every lane evaluates
// its queued pairs and sums its own target -- so the pair arithmetic runs for
// in-range pairs only, with the warp's lanes busy, and no atomics.  r from the
// wrapped FP64 positions and the image shift of the cell offset, the cutoff
// and the pair in FP64 (R = double).
template <typename R>
__global__ void __launch_bounds__(kDlWarps * 32) k_p2p_dl(DlNearArgs a)
{
    __shared__ DlQueue wq[kDlWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DlQueue &w = wq[warp];
    const int64_t t = ((int64_t)blockIdx.x * kDlWarps + warp) * 32 + lane;
    const bool active = t < a.N;
    const int nc = a.nc, K = a.K, side = 2 * K + 1, nO = side * side * side;
    int i = 0, cx = 0, cy = 0, cz = 0;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
    if (active) {
        i = a.permn[t];
        const int c = a.keyn[i] / kSub3;
        cx = c % nc;
        cy = (c / nc) % nc;
        cz = c / (nc * nc);
        th = a.lhi[t];
        tl = a.llo[t];
    }
    // walk state: next neighbour offset oi, current source range [s, se) of
    // the neighbour cell at offset (ox, oy, oz), and the target relative to it
    int oi = active ? 0 : nO, s = 0, se = 0, code = 0;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
    auto next_cell = [&]() {
        while (s == se && oi < nO) {
            const int ox = oi % side - K, oy = (oi / side) % side - K, oz = oi / (side * side) - K;
            ++oi;
            const int ax = cx + ox, ay = cy + oy, az = cz + oz;
            const int bx = ax - floor_div(ax, nc) * nc, by = ay - floor_div(ay, nc) * nc,
                      bz = az - floor_div(az, nc) * nc;
            const int nb = (bz * nc + by) * nc + bx;
            s = a.startn[nb * kSub3];
            se = a.startn[(nb + 1) * kSub3];
            code = (ox + 64) | ((oy + 64) << 8) | ((oz + 64) << 16);
            b0 = th.x - (float)ox;  // exact: th on the 2^-20 lattice
            b1 = th.y - (float)oy;
            b2 = th.z - (float)oz;
        }
    };
    next_cell();
    const R xi = (R)a.xi, c_e = (R)(2.0 * a.xi / 1.7724538509055160273);  // 2 xi / sqrt(pi)
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    if constexpr (sizeof(R) == 8) {
        if (active) {
            const dvec4 P = a.pos[t];
            t0 = P.x;
            t1 = P.y;
            t2 = P.z;
        }
    }
    int len = 0;
    auto evaluate = [&]() {
        const int m = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
        R v0 = 0, v1 = 0, v2 = 0;
        for (int k = 0; k < m; ++k) {
            if (k < len) {
                const int sj = w.src[k][lane], cd = w.code[k][lane];
                const int ox = (cd & 255) - 64, oy = ((cd >> 8) & 255) - 64, oz = ((cd >> 16) & 255) - 64;
                const int sx = floor_div(cx + ox, nc), sy = floor_div(cy + oy, nc), sz = floor_div(cz + oz, nc);
                const dvec4 P = a.pos[sj];
                const double r0 = (t0 - a.L * sx) - P.x, r1 = (t1 - a.L * sy) - P.y, r2 = (t2 - a.L * sz) - P.z;
                const double rr2 = fma(r0, r0, fma(r1, r1, r2 * r2));
                if (rr2 <= a.rc2 && rr2 > 0.0) {
                    const dvec4 Q = a.qs[sj], Nn = a.ns[sj];
                    dl_pair<double>(r0, r1, r2, rr2, Q.x, Q.y, Q.z, Nn.x, Nn.y, Nn.z, xi, c_e, v0, v1, v2);
                }
            }
        }
        u0 += (double)v0;
        u1 += (double)v1;
        u2 += (double)v2;
        len = 0;
    };
    while (__any_sync(0xffffffffu, s < se)) {
        if (s < se) {
            const float4 P = a.lhi[s];
            const float r0 = b0 - P.x, r1 = b1 - P.y, r2 = b2 - P.z;
            if (fmaf(r0, r0, fmaf(r1, r1, r2 * r2)) <= a.rcm2) {
                w.src[len][lane] = s;
                w.code[len][lane] = code;
                ++len;
            }
            ++s;
            next_cell();
        }
        if (__any_sync(0xffffffffu, len == kDlQ))
            evaluate();
    }
    evaluate();
    if (active) {
        a.u[3 * i] += u0;
        a.u[3 * i + 1] += u1;
        a.u[3 * i + 2] += u2;
    }
}

// Double-layer source records for the FP32 near field (k_p2p_dl32), near
// order: the cell-local position parts of the slot's Stokeslet record (lo and
// the packed 2^-20 lattice hi) and the symmetric part S of q (x) n in FP32:
//   (lo.x, lo.y, lo.z, S_xx), (S_yy, S_zz, hi bits 0..31, hi bits 32..63),
//   (S_xy, S_xz, S_yz, 0).
__global__ void __launch_bounds__(256) k_dl_records(const double *__restrict__ q, const double *__restrict__ n,
                                                    const int32_t *__restrict__ permn,
                                                    const float4 *__restrict__ nrec, int64_t N,
                                                    float4 *__restrict__ drec, int *err)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N)
        return;
    const int64_t j = permn[s];
    const double q0 = q[3 * j], q1 = q[3 * j + 1], q2 = q[3 * j + 2];
    const double n0 = n[3 * j], n1 = n[3 * j + 1], n2 = n[3 * j + 2];
    if (!(isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(n0) && isfinite(n1) && isfinite(n2)))
        atomicOr(err, 1);
    const float4 A = nrec[2 * s], B = nrec[2 * s + 1];
    drec[3 * s] = make_float4(A.x, A.y, A.z, (float)(q0 * n0));
    drec[3 * s + 1] = make_float4((float)(q1 * n1), (float)(q2 * n2), B.z, B.w);
    drec[3 * s + 2] = make_float4((float)(0.5 * (q0 * n1 + q1 * n0)), (float)(0.5 * (q0 * n2 + q2 * n0)),
                                  (float)(0.5 * (q1 * n2 + q2 * n1)), 0.f);
}

}  // namespace

cudaError_t launch_dl_records(ewald_plan_s *p, const double *q, const double *n, void *drec, cudaStream_t s)
{
    const int64_t N = p->N;
    k_dl_records<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(q, n, p->permn, (const float4 *)p->nrec, N,
                                                             (float4 *)drec, p->err);
    return cudaGetLastError();
}

cudaError_t launch_dl_densities(ewald_plan_s *p, const double *q, const double *n, cudaStream_t s)
{
    const int64_t N = p->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (p->grid_ds) {  // two float4 per point and triple (64 bytes a point in all)
        float4 *sd = (float4 *)p->dl_tf;
        k_dl_densities_ds<<<nb, 256, 0, s>>>(q, n, p->permt, N, sd, sd + 2 * N, p->err);
    } else if (p->near64) {
        dvec4 *sd = (dvec4 *)p->dl_tf;
        k_dl_densities<dvec4><<<nb, 256, 0, s>>>(q, n, p->permt, N, sd, sd + N, p->err);
    } else {
        float4 *sd = (float4 *)p->dl_tf;
        k_dl_densities<float4><<<nb, 256, 0, s>>>(q, n, p->permt, N, sd, sd + N, p->err);
    }
    return cudaGetLastError();
}

cudaError_t launch_scale_dl(ewald_plan_s *p, double C, cudaStream_t s)
{
    const double kfac = 2.0 * 3.14159265358979323846 / p->prm.L;
    const double inv4xi2 = 1.0 / (4.0 * p->prm.xi * p->prm.xi);
    const int64_t n = p->g.ncplx;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (p->fft64) {
        const double2 *sa = (const double2 *)p->dl_spec;
        k_scale_dl<double, double2><<<nb, 256, 0, s>>>((double2 *)p->spec, sa, sa + 3 * n,
                                                       (const double *)p->tab, p->g.M, p->g.Mh, n, kfac,
                                                       inv4xi2, C);
    } else {
        const float2 *sa = (const float2 *)p->dl_spec;
        k_scale_dl<float, float2><<<nb, 256, 0, s>>>((float2 *)p->spec, sa, sa + 3 * n, (const float *)p->tab,
                                                     p->g.M, p->g.Mh, n, (float)kfac, (float)inv4xi2,
                                                     (float)C);
    }
    return cudaGetLastError();
}

cudaError_t launch_p2p_dl(ewald_plan_s *p, const double *x, const double *q, const double *n, double *u,
                          cudaStream_t s)
{
    const int64_t N = p->N;
    dvec4 *pos = (dvec4 *)p->dl_near, *qs = pos + N, *ns = qs + N;
    float4 *lhi = (float4 *)(ns + N), *llo = lhi + N, *q32 = llo + N, *n32 = q32 + N;
    k_dl_sort<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(x, q, n, p->permn, p->keyn, N, p->prm.L, 1.0 / p->prm.L,
                                                          1.0 / p->g.cell, p->g.nc, pos, qs, ns, lhi, llo, q32, n32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    DlNearArgs a;
    a.permn = p->permn;
    a.keyn = p->keyn;
    a.startn = p->startn;
    a.pos = pos;
    a.qs = qs;
    a.ns = ns;
    a.lhi = lhi;
    a.llo = llo;
    a.q32 = q32;
    a.n32 = n32;
    a.u = u;
    a.N = N;
    a.L = p->prm.L;
    a.xi = p->prm.xi;
    a.rc2 = p->prm.rc * p->prm.rc;
    a.w = (float)p->g.cell;
    // the filter works on the hi parts alone, in cell units: each is within
    // 2^-21 of its coordinate, so a margin of 1e-4 rc + 1e-5 cell covers it
    const double rcm = (p->prm.rc / p->g.cell) * (1.0 + 1e-4) + 1e-5;
    a.rcm2 = (float)(rcm * rcm);
    a.nc = p->g.nc;
    a.K = p->g.K;
    const unsigned nb = (unsigned)((N + 32 * kDlWarps - 1) / (32 * kDlWarps));
    // FP64 pairs (plans with FP64 FFTs or FP64 kernels; FP32 plans take
    // k_p2p_dl32 in k_p2p.cu)
    k_p2p_dl<double><<<nb, 32 * kDlWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ewg
