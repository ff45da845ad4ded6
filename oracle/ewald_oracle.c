/*
 * ewald_oracle.c -- plain CPU FP64 reference for the triply periodic
 * Stokeslet sum (Kosmacher, Du, Bagge, Biros, "A Performance Portable Fast
 * Ewald Summation for Stokes Flow").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (Sec. 2: the periodized sum eq. (potentials), split by
 * Sec. 2.1-2.2, with the fully periodic reading of the image set):
 *
 *   u_i = sum_j sum'_{p in L Z^3} G^N(x_i - x_j + p) f_j
 *       + (1/L^3) sum_{k != 0} Re[ Ghat^F(k) S(k) e^{i k.x_i} ]
 *       - (4 xi / sqrt(pi)) sum_{j : x_j = x_i} f_j,   S(k) = sum_j f_j e^{-i k.x_j}
 *
 * with G(r) = I/|r| + r r^T/|r|^3 (no 1/(8 pi mu) factor, Sec. 2), the
 * Hasimoto near-field kernel G^N of eq. (g-near) and the far-field transform
 * Ghat^F of eq. (GFk).  The prime drops every pair at r = 0: Sec. 2 skips the
 * term of a point at the target's position, and skipping the whole G term
 * means also removing its far part G^F(0) f_j = (4 xi / sqrt(pi)) f_j, which
 * the k sum holds; for j = i that is the usual self term lim_{r->0}(G - G^N).
 * Removing it for distinct coincident points too keeps the result
 * independent of xi.  The k = 0 mode is dropped (zero mean velocity,
 * Hasimoto's convention).
 *
 * Truncation: real space keeps |r| < sqrt(40)/xi (erfc(sqrt 40) ~ 4e-19),
 * k space keeps |k| < 2 xi sqrt(40) (Gaussian factor e^{-40}), so for any xi
 * the result is the converged lattice sum to FP64 rounding.  Sums use
 * Neumaier compensation.  All loops run in the order the definitions state;
 * OpenMP only splits independent targets or independent wave vectors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ---- compensated (Neumaier) summation ---------------------------------- */
typedef struct { double s, c; } csum;

static inline void cadd(csum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}
static inline double cval(const csum *a) { return a->s + a->c; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- kernels written as the paper prints them -------------------------- */

/* Stokeslet G(r) = I/|r| + r r^T / |r|^3   (Sec. 2). */
static void stokeslet(const double r[3], double G[3][3])
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            G[a][b] = (a == b ? 1.0 / rn : 0.0) + r[a] * r[b] / (r2 * rn);
}

/* Near-field Stokeslet, Sec. 2.1 eq. (g-near):
 *   G^N(r) = G(r) ( erfc(xi|r|) + 2 xi |r| e^{-xi^2|r|^2}/sqrt(pi) )
 *            - I 4 xi e^{-xi^2 |r|^2} / sqrt(pi)                          */
static void near_stokeslet(const double r[3], double xi, double GN[3][3])
{
    double G[3][3];
    stokeslet(r, G);
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double e = exp(-xi * xi * rn * rn);
    double bracket = erfc(xi * rn) + rn * 2.0 * xi * e / sqrt(ORACLE_PI);
    double diag = 4.0 * xi * e / sqrt(ORACLE_PI);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            GN[a][b] = G[a][b] * bracket - (a == b ? diag : 0.0);
}

/* Far-field transform, Sec. 2.2 eq. (GFk):
 *   Ghat^F(k) = 8 pi / |k|^4 (I |k|^2 - k k^T) e^{-|k|^2/(2xi)^2}
 *               (1 + |k|^2/(2xi)^2)                                        */
static void far_stokeslet_hat(const double k[3], double xi, double Gh[3][3])
{
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double q = k2 / (4.0 * xi * xi);
    double s = 8.0 * ORACLE_PI / (k2 * k2) * exp(-q) * (1.0 + q);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Gh[a][b] = s * ((a == b ? k2 : 0.0) - k[a] * k[b]);
}

/* Integer image range along one axis: all a with |d + a L| < R
 * (d = x_i - x_j along that axis).  Exact enumeration of the images whose
 * coordinate difference can lie inside the sphere of radius R. */
static void image_range(double d, double L, double R, long *lo, long *hi)
{
    *lo = (long)ceil((-R - d) / L);
    *hi = (long)floor((R - d) / L);
}

/* Sum over j and images p of G^N(x_t - x_j + p) f_j for 0 < |r| < R (open)
 * or 0 < |r| <= R (closed).  A pair at r = 0 (the point itself, or a
 * distinct point at the same position) is skipped as a whole, Sec. 2: its
 * near part is left out here, and its far part, which the k-space sum
 * contains as G^F(0) f_j = (4 xi / sqrt(pi)) f_j, is taken out here too --
 * for j = i this is the usual self term. */
static void real_space_target(int64_t n, double L, const double *x,
                              const double *f, const double *xt, double R,
                              int closed, double xi, double out[3])
{
    const double self = 4.0 * xi / sqrt(ORACLE_PI);
    csum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t j = 0; j < n; ++j) {
        double d[3];
        long lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            d[a] = xt[a] - x[3 * j + a];
            image_range(d[a], L, R, &lo[a], &hi[a]);
        }
        for (long p0 = lo[0]; p0 <= hi[0]; ++p0)
            for (long p1 = lo[1]; p1 <= hi[1]; ++p1)
                for (long p2 = lo[2]; p2 <= hi[2]; ++p2) {
                    double r[3] = {d[0] + p0 * L, d[1] + p1 * L, d[2] + p2 * L};
                    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (r2 == 0.0) { /* self or coincident: whole term skipped */
                        for (int a = 0; a < 3; ++a)
                            cadd(&acc[a], -self * f[3 * j + a]);
                        continue;
                    }
                    if (closed ? (r2 > R * R) : (r2 >= R * R))
                        continue;
                    double K[3][3];
                    near_stokeslet(r, xi, K);
                    for (int a = 0; a < 3; ++a)
                        cadd(&acc[a], K[a][0] * f[3 * j + 0] +
                                          K[a][1] * f[3 * j + 1] +
                                          K[a][2] * f[3 * j + 2]);
                }
    }
    for (int a = 0; a < 3; ++a)
        out[a] = cval(&acc[a]);
}

/* ---- k space ------------------------------------------------------------ */

/* Wave vectors k = 2 pi m / L, m != 0.  kbox > 0: |m_d| <= kbox per axis;
 * kbox <= 0: the sphere |k| < 2 xi sqrt(40).  Returns a malloc'd list. */
static int64_t wave_vectors(double L, double xi, int64_t kbox, double **out)
{
    double kcut = 2.0 * xi * sqrt(40.0);
    long mmax = kbox > 0 ? (long)kbox : (long)ceil(kcut * L / (2.0 * ORACLE_PI));
    int64_t cap = (int64_t)(2 * mmax + 1) * (2 * mmax + 1) * (2 * mmax + 1);
    double *k = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
    if (!k)
        return -1;
    int64_t nk = 0;
    for (long m0 = -mmax; m0 <= mmax; ++m0)
        for (long m1 = -mmax; m1 <= mmax; ++m1)
            for (long m2 = -mmax; m2 <= mmax; ++m2) {
                if (m0 == 0 && m1 == 0 && m2 == 0)
                    continue; /* k = 0 dropped */
                double kv[3] = {2.0 * ORACLE_PI * m0 / L, 2.0 * ORACLE_PI * m1 / L,
                                2.0 * ORACLE_PI * m2 / L};
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
                if (kbox <= 0 && k2 >= kcut * kcut)
                    continue;
                k[3 * nk + 0] = kv[0];
                k[3 * nk + 1] = kv[1];
                k[3 * nk + 2] = kv[2];
                ++nk;
            }
    *out = k;
    return nk;
}

/* Far field at the targets: (1/L^3) sum_k Re[Ghat^F(k) S(k) e^{i k.x_t}]. */
static int far_field(int64_t n, double L, const double *x, const double *f,
                     double xi, int64_t kbox, int64_t nt, const double *xt,
                     double *u)
{
    double *k = NULL;
    int64_t nk = wave_vectors(L, xi, kbox, &k);
    if (nk < 0)
        return -1;
    /* structure factor S(k) = sum_j f_j e^{-i k.x_j}: 3 complex per k */
    double *S = (double *)malloc(sizeof(double) * 6 * (size_t)(nk > 0 ? nk : 1));
    if (!S) {
        free(k);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nk; ++q) {
        csum re[3] = {{0, 0}, {0, 0}, {0, 0}}, im[3] = {{0, 0}, {0, 0}, {0, 0}};
        const double *kv = &k[3 * q];
        for (int64_t j = 0; j < n; ++j) {
            double ph = -(kv[0] * x[3 * j] + kv[1] * x[3 * j + 1] + kv[2] * x[3 * j + 2]);
            double c = cos(ph), s = sin(ph);
            for (int a = 0; a < 3; ++a) {
                cadd(&re[a], f[3 * j + a] * c);
                cadd(&im[a], f[3 * j + a] * s);
            }
        }
        for (int a = 0; a < 3; ++a) {
            S[6 * q + 2 * a] = cval(&re[a]);
            S[6 * q + 2 * a + 1] = cval(&im[a]);
        }
    }
    double V = L * L * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nt; ++t) {
        csum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t q = 0; q < nk; ++q) {
            const double *kv = &k[3 * q];
            double Gh[3][3];
            far_stokeslet_hat(kv, xi, Gh);
            double ph = kv[0] * xt[3 * t] + kv[1] * xt[3 * t + 1] + kv[2] * xt[3 * t + 2];
            double c = cos(ph), s = sin(ph);
            for (int a = 0; a < 3; ++a) {
                /* Re[(sum_b Gh[a][b] S_b) e^{i ph}] */
                double vr = 0.0, vi = 0.0;
                for (int b = 0; b < 3; ++b) {
                    vr += Gh[a][b] * S[6 * q + 2 * b];
                    vi += Gh[a][b] * S[6 * q + 2 * b + 1];
                }
                cadd(&acc[a], (vr * c - vi * s) / V);
            }
        }
        for (int a = 0; a < 3; ++a)
            u[3 * t + a] = cval(&acc[a]);
    }
    free(S);
    free(k);
    return 0;
}

static void gather_targets(const double *x, int64_t nt, const int64_t *tidx, double *xt)
{
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a)
            xt[3 * t + a] = x[3 * (tidx ? tidx[t] : t) + a];
}

/* ---- exported entry points ----------------------------------------------- */

/* Full direct Ewald sum at nt targets (indices tidx into x; NULL = all n).
 * u: nt x 3.  Returns 0 on success, -1 on allocation failure. */
int oracle_ewald(int64_t n, double L, const double *x, const double *f, double xi,
                 int64_t nt, const int64_t *tidx, double *u)
{
    double *xt = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    double *uf = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    if (!xt || !uf) {
        free(xt);
        free(uf);
        return -1;
    }
    gather_targets(x, nt, tidx, xt);
    double R = sqrt(40.0) / xi;
    if (far_field(n, L, x, f, xi, 0, nt, xt, uf) != 0) {
        free(xt);
        free(uf);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nt; ++t) {
        double un[3];
        real_space_target(n, L, x, f, &xt[3 * t], R, 0, xi, un); /* includes the self term */
        for (int a = 0; a < 3; ++a)
            u[3 * t + a] = un[a] + uf[3 * t + a];
    }
    free(xt);
    free(uf);
    return 0;
}

/* Near field (the P2P stage, Sec. 2.1 eq. (potentials-near)): sum over j and
 * images with 0 < |r| <= rc of G^N(r) f_j, minus (4 xi/sqrt(pi)) f_j for
 * every pair at r = 0 (self and coincident points), at every point.  u: n x 3. */
int oracle_near_field(int64_t n, double L, const double *x, const double *f,
                      double xi, double rc, double *u)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < n; ++t)
        real_space_target(n, L, x, f, &x[3 * t], rc, 1, xi, &u[3 * t]);
    return 0;
}

/* Far field only, by direct k sum (Sec. 2.2 eq. (potentials-far), (GFk),
 * with a Fourier series in all three periodic directions), at nt targets; no self term is removed.  kbox > 0 restricts the
 * wave numbers to |m_d| <= kbox (the k set a grid of size 2 kbox + 2 holds
 * without its Nyquist planes); kbox <= 0 uses the converged sphere. */
int oracle_far_field(int64_t n, double L, const double *x, const double *f,
                     double xi, int64_t kbox, int64_t nt, const int64_t *tidx,
                     double *u)
{
    double *xt = (double *)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    if (!xt)
        return -1;
    gather_targets(x, nt, tidx, xt);
    int rc = far_field(n, L, x, f, xi, kbox, nt, xt, u);
    free(xt);
    return rc;
}

/* Brute-force spherical image sum of the bare Stokeslet over whole periodic
 * cells:  u_i = sum_{p in L Z^3, |p| < R} sum_j G(x_i - x_j + p) f_j, skipping
 * r = 0.  Each cell is complete, so a force-free cell adds no monopole; the
 * lattice sum is still only conditionally convergent, and as R grows it tends
 * to the Ewald value plus an affine field c + A x_i (the surface term of the
 * spherical summation order). */
int oracle_image_sum(int64_t n, double L, const double *x, const double *f,
                     double R, double *u)
{
    long m = (long)ceil(R / L);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < n; ++t) {
        csum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (long p0 = -m; p0 <= m; ++p0)
            for (long p1 = -m; p1 <= m; ++p1)
                for (long p2 = -m; p2 <= m; ++p2) {
                    double p[3] = {p0 * L, p1 * L, p2 * L};
                    if (p[0] * p[0] + p[1] * p[1] + p[2] * p[2] >= R * R)
                        continue;
                    for (int64_t j = 0; j < n; ++j) {
                        double r[3];
                        for (int a = 0; a < 3; ++a)
                            r[a] = x[3 * t + a] - x[3 * j + a] + p[a];
                        if (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] == 0.0)
                            continue;
                        double G[3][3];
                        stokeslet(r, G);
                        for (int a = 0; a < 3; ++a)
                            cadd(&acc[a], G[a][0] * f[3 * j + 0] + G[a][1] * f[3 * j + 1] +
                                              G[a][2] * f[3 * j + 2]);
                    }
                }
        for (int a = 0; a < 3; ++a)
            u[3 * t + a] = cval(&acc[a]);
    }
    return 0;
}
