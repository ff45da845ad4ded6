// params.cpp -- host-only math of the planner: Bessel I0, the truncated
// Kaiser-Bessel window and its transform, the piecewise-polynomial window fit,
// and the parameter choice from the error estimate eq. (ese).  No CUDA calls.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "erf_rational.h"
#include "internal.h"

namespace ewg {

static const double kPi = 3.14159265358979323846;
// Plain FP32 serves tolerances above this; tol = 1e-7 itself is below (the
// floor sits a rounding above 1e-7 so that the literal 1e-7 selects it).
static const double kFp32TolFloor = 1.0000001e-7;

// Modified Bessel function I0 by its power series sum_k ((x/2)^{2k}) / (k!)^2;
// all terms are positive, so the sum is accurate to rounding for any x.
double bessel_i0(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum)
            break;
    }
    return sum;
}

// Truncated Kaiser-Bessel window of Sec. 2.2 with beta = 2.5 P, a_w = P h / 2,
// written in grid units t = r / h:  I0(beta sqrt(1 - (2t/P)^2)) / I0(beta)
// for |t| < P/2, else 0.
double kb_window(double t, int P)
{
    double half = 0.5 * P;
    if (fabs(t) >= half)
        return 0.0;
    double beta = 2.5 * P;
    double s = t / half;
    return bessel_i0(beta * sqrt(1.0 - s * s)) / bessel_i0(beta);
}

// Transform of the truncated window, int w_0(r) e^{-ikr} dr (used in eq. (sca),
// where the paper leaves it implicit): with a = a_w, s^2 = beta^2 - (k a)^2,
// 2a sinh(s)/(s I0(beta)); past k a = beta the sinh turns into a sin.
double kb_window_hat(double k, double h, int P)
{
    double beta = 2.5 * P, a = 0.5 * P * h;
    double d = beta * beta - (k * a) * (k * a);
    double i0b = bessel_i0(beta);
    if (d > 0) {
        double s = sqrt(d);
        return 2.0 * a * sinh(s) / (s * i0b);
    }
    if (d < 0) {
        double s = sqrt(-d);
        return 2.0 * a * sin(s) / (s * i0b);
    }
    return 2.0 * a / i0b;
}

// Piecewise-polynomial window (Sec. 2.2 and Sec. 4): for a point whose
// fractional grid offset is delta in [0, 1), the P window values are
// w_l(delta) = w_0(l + 1 - P/2 - delta), l = 0..P-1 (one bin of width h each).
// Each bin is interpolated at deg+1 Chebyshev nodes in z = 2 delta - 1 and
// stored as monomial coefficients in z for Horner evaluation.
ewald_status fit_window(int P, int deg, WindowPoly *out, double *max_err)
{
    if (P < 2 || P > kMaxP || deg < 1 || deg > kMaxDeg)
        return EWALD_EUNSUPPORTED;
    int n = deg + 1;
    out->P = P;
    out->deg = deg;
    out->coef.assign((size_t)P * n, 0.0);
    std::vector<double> znode(n), cheb(n), Tprev(n), Tcur(n), Tnext(n), mono(n);
    for (int j = 0; j < n; ++j)
        znode[j] = cos(kPi * (j + 0.5) / n);
    double worst = 0.0;
    for (int l = 0; l < P; ++l) {
        auto g = [&](double z) { return kb_window(l + 1 - 0.5 * P - 0.5 * (z + 1.0), P); };
        // Chebyshev coefficients c_m = (2/n) sum_j g(z_j) T_m(z_j), c_0 halved
        for (int m = 0; m < n; ++m) {
            double s = 0.0;
            for (int j = 0; j < n; ++j)
                s += g(znode[j]) * cos(m * kPi * (j + 0.5) / n);
            cheb[m] = (m == 0 ? 1.0 : 2.0) * s / n;
        }
        // monomial form: accumulate c_m T_m(z) with T_{m+1} = 2 z T_m - T_{m-1}
        std::fill(mono.begin(), mono.end(), 0.0);
        std::fill(Tprev.begin(), Tprev.end(), 0.0);
        std::fill(Tcur.begin(), Tcur.end(), 0.0);
        Tprev[0] = 1.0;                  // T_0
        if (n > 1)
            Tcur[1] = 1.0;               // T_1
        for (int k = 0; k < n; ++k)
            mono[k] += cheb[0] * Tprev[k];
        for (int m = 1; m < n; ++m) {
            for (int k = 0; k < n; ++k)
                mono[k] += cheb[m] * Tcur[k];
            std::fill(Tnext.begin(), Tnext.end(), 0.0);
            for (int k = 0; k < n; ++k) {
                if (k + 1 < n)
                    Tnext[k + 1] += 2.0 * Tcur[k];
                Tnext[k] -= Tprev[k];
            }
            Tprev = Tcur;
            Tcur = Tnext;
        }
        for (int k = 0; k < n; ++k)
            out->coef[(size_t)l * n + k] = mono[k];
        // dense check of the monomial form against the exact window, on the
        // open bin (at |t| = P/2 the truncated window jumps from 1/I0(beta)
        // to 0; the fit takes the one-sided limit there)
        for (int i = 0; i <= 256; ++i) {
            double z = -1.0 + 2.0 * (i + 0.5) / 257.0;
            double p = 0.0;
            for (int k = n - 1; k >= 0; --k)
                p = p * z + mono[k];
            worst = std::max(worst, fabs(p - g(z)));
        }
    }
    if (max_err)
        *max_err = worst;
    return EWALD_OK;
}

// ---- error estimate eq. (ese), unit box, unit sum |f|^2 --------------------
static double est_near(double xi, double rc)
{
    return sqrt(112.0 / 9.0 * pow(xi, 4) * pow(rc, 3)) * exp(-xi * xi * rc * rc);
}
static double est_far(double h, double xi)
{
    return 4.0 / (3.0 * h) * sqrt(3.5) * exp(-kPi * kPi / pow(2.0 * h * xi, 2));
}
// E^w = C(xi) e^{-2.5 P}; the paper leaves C(xi) open.  Measured with the
// exact window against the direct k sum on the grid's k set: C ~ 20 while
// h xi is small, and an aliasing floor ~ 5e-4 e^{-0.95 P} near h xi ~ 0.33,
// where the selection rule below puts it.
static double est_window(int P)
{
    return 20.0 * exp(-2.5 * P) + 5e-4 * exp(-0.95 * P);
}
// largest xi with E^F(h, xi) <= target
static double xi_for_grid(double h, double target)
{
    double lg = log(4.0 / (3.0 * h) * sqrt(3.5) / target);
    if (lg <= 0)
        lg = 1e-3;
    return kPi / (2.0 * h * sqrt(lg));
}
// smallest rc with E^N(xi, rc) <= target (E^N decreases for xi rc > 1.3)
static double rc_for_xi(double xi, double target)
{
    double lo = 1.3 / xi, hi = 12.0 / xi;
    if (est_near(xi, lo) <= target)
        return lo;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (est_near(xi, mid) <= target)
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}
// cuFFT's relative cost per element for sizes with a radix-7 or radix-5 factor
// (measured, FP64 3-D real transforms on GB300: M = 112 ran ~40 % and M = 160
// ~20 % above the m^3 log m^3 scaling of M = 128 and 144)
static double fft_size_factor(int m)
{
    return 1.0 + (m % 7 == 0 ? 0.4 : 0.0) + (m % 5 == 0 ? 0.2 : 0.0);
}

static bool fft_friendly(int m)
{
    if (m % 2)
        return false;
    for (int p : {2, 3, 5, 7})
        while (m % p == 0)
            m /= p;
    return m == 1;
}

// Split radius of the double-single near field (FP32-bulk plans at tol <=
// 1e-7).  A pair's term is G^N(r) f, |G^N f|^2 averaged over directions of f
// = |f|^2 (2 (A - B)^2 + 4 A^2) / 3 with A = erfc(x)/r, B = (2 xi/sqrt(pi))
// e^{-x^2}, x = xi r (eq. (g-near)); its size falls off with x.  Pairs beyond
// r1 = x1/xi are evaluated in the two-pair FP32 bulk form with compensated
// sums, those within r1 in double-single.  The bulk form's relative error per
// term is eps(x) = sqrt(eps0^2 + (eps1 x^2)^2): eps0 = 3e-7 from the erfcx fit
// and the hardware rsqrt, ex2 and rcp approximations, and eps1 x^2 (eps1 =
// 1.2e-7) from e^{-x^2} = 2^a with a = -x^2 log2(e) computed from the FP32
// r^2 (two units in the last place of a, times |a| ln 2).  Their random
// errors add to ~sqrt(sum over the pairs beyond r1 of eps^2 |term|^2); x1 is
// the smallest x for which, with pairs spread uniformly in space (density ~
// x^2: the case with the most weight beyond x1; clustered points put more of
// it close), that sum stays below (tol/5)^2 sum |term|^2 -- the FP32 part's
// error then stays near tol/5 of the near field, which with the three eq.
// (ese) terms held at tol/10 each keeps the total within tol.  Returns rc
// when nothing is left to split off.
double ds_split_radius(double tol, double xi, double rc)
{
    const double xc = xi * rc;
    if (!(xc > 0) || !(tol > 0))
        return rc;
    constexpr double eps0 = 3e-7, eps1 = 1.2e-7;
    const double target = (tol / 5.0) * (tol / 5.0);
    auto w = [](double x) {
        if (x <= 0.0)
            return 6.0;  // the limit x^2 (2 (A - B)^2 + 4 A^2) as x -> 0 (units of xi |f|)
        const double A = erfc(x) / x, B = 1.1283791670955126 * exp(-x * x);
        return x * x * (2.0 * (A - B) * (A - B) + 4.0 * A * A);
    };
    auto ew = [&](double x) { return (eps0 * eps0 + eps1 * eps1 * x * x * x * x) * w(x); };
    // composite Simpson on n panels, accumulated from xc down
    const int n = 4000;
    const double hx = xc / n;
    std::vector<double> tail(n + 1, 0.0);  // tail[i] = integral of eps^2 w from x_i to xc
    double total = 0.0;                     // integral of w from 0 to xc
    for (int i = n - 1; i >= 0; --i) {
        const double a = i * hx, b = a + hx, m = 0.5 * (a + b);
        tail[i] = tail[i + 1] + hx / 6.0 * (ew(a) + 4.0 * ew(m) + ew(b));
        total += hx / 6.0 * (w(a) + 4.0 * w(m) + w(b));
    }
    if (tail[0] <= target * total)
        return 0.0;  // the bulk form holds everywhere: nothing to split off
    for (int i = 0; i <= n; ++i)
        if (tail[i] <= target * total)
            return i >= n ? rc : (i * hx) / xi;
    return rc;
}

ewald_status choose_params(int64_t N, double L, double tol, ewald_dtype dtype,
                           const ewald_params *ov, ewald_params *out)
{
    if (!out || N < 1 || !(L > 0) || !std::isfinite(L) || !(tol >= 1e-12 && tol <= 1e-2))
        return EWALD_EINVAL;
    if (dtype != EWALD_F64 && dtype != EWALD_F32_BULK)
        return EWALD_EINVAL;
    ewald_params o;
    memset(&o, 0, sizeof(o));
    if (ov)
        o = *ov;
    ewald_params p;
    memset(&p, 0, sizeof(p));
    p.L = L;
    p.tol = tol;
    // Plain FP32 pair and grid arithmetic reaches tol 1e-6 with margin but
    // not 1e-7: on the clustered 2e6 workload (tol 1e-7, M = 256, P = 14) the
    // FP32 near field's max error over all points was 1.03e-7 of max |u| and
    // the FP32 grid's rms error 7.8e-8 (measured against the FP64 kernels).
    // So at tol <= 1e-7 the FP32-bulk P2P runs in double-single arithmetic
    // (the FP64 pipe is 1/64 of the FP32 one on this GPU), down to 1e-9, and
    // P2G/G2P in double-single or FP64 (near_f64 marks both).
    const bool below_fp32 = tol < kFp32TolFloor;
    p.near_f64 = (dtype == EWALD_F64 || below_fp32) ? 1 : 0;
    p.near_ds = (dtype == EWALD_F32_BULK && below_fp32 && tol >= 1e-9) ? 1 : 0;
    p.fft_f64 = (dtype == EWALD_F64 || tol < 1e-6) ? 1 : 0;
    // each estimated term held to tol/10: the estimate is an rms for unit
    // sum |f|^2, and the max-norm error runs about 3x the rms one (measured)
    const double target = tol / 10.0;

    // window support P (Sec. 2.2): smallest with E^w <= target
    int P = o.P;
    if (P <= 0) {
        P = 3;
        while (P < kMaxP && est_window(P) > target)
            ++P;
    }
    if (P < 2 || P > kMaxP)
        return EWALD_EUNSUPPORTED;

    // Work in the unit box: xi' = xi L, rc' = rc / L, h' = h / L.
    double xi = o.xi > 0 ? o.xi * L : 0.0;
    double rc = o.rc > 0 ? o.rc / L : 0.0;
    int M = o.M;
    if (M > 0) {
        if (xi <= 0)
            xi = xi_for_grid(1.0 / M, target);
    } else if (xi > 0) {
        // smallest friendly M with E^F <= target at the given xi
        M = 8 * ((std::max(8, P + 2) + 7) / 8);
        while (M < 4096 && (!fft_friendly(M) || est_far(1.0 / M, xi) > target))
            M += 8;
    } else {
        // minimise a per-stage cost model over friendly grid sizes
        double best = 1e300;
        for (int m = 8 * ((std::max(8, P + 2) + 7) / 8); m <= 1024; m += 8) {
            if (!fft_friendly(m))
                continue;
            double x = xi_for_grid(1.0 / m, target);
            double r = rc_for_xi(x, target);
            int nc = std::max(1, (int)floor(1.0 / r));
            double cellv = pow(1.0 / nc, 3);
            double cand = (double)N * (double)N * 27.0 * cellv;       // P2P candidates
            double inr = (double)N * (double)N * 4.18879 * r * r * r;  // in-range pairs
            double m3 = (double)m * m * m;
            // stage weights fitted to GB300 stage times (FP32: N = 1e5, M =
            // 128, P = 12: P2P 0.34, P2G + G2P 0.35, FFTs + CNV 0.10 ms;
            // double-single and FP64: N = 1e4 .. 1e6 over a range of M): one
            // unit ~5.3e-11 ms.  The FP64 pipe is 1/64 of the FP32 one, so
            // FP64 plans move work from the near field to the grid.  The
            // split double-single near field measured 1.8-2.6x the FP32 work
            // rate (N = 1e5 and 1e6, tol 1e-8, M = 72 .. 392).
            const double wn = p.near_ds ? 2.5 : (p.near_f64 ? 48.0 : 1.0);
            const double wg = p.near_ds ? 3.65 : (p.near_f64 ? 13.6 : 1.0);
            const double wf = p.fft_f64 ? 26.0 : 1.55;
            const double halo = pow((8.0 + P - 1.0) / 8.0, 3);      // staged block / tile
            double cost = wn * (10.0 * cand + 50.0 * inr)              // P2P
                          + wg * 28.0 * (double)N * P * P * P          // P2G + G2P per point
                          + wg * 65.0 * m3 * halo                      // P2G + G2P per tile
                          + wf * 27.0 * m3 * log2(m3) * fft_size_factor(m);  // FFTs
            if (cost < best) {
                best = cost;
                M = m;
                xi = x;
            }
        }
    }
    if (M < 4 || M > 4096 || M < P)
        return EWALD_EUNSUPPORTED;
    if (rc <= 0)
        rc = rc_for_xi(xi, target);
    // cell list: n_c = floor(L / rc) cells of width >= rc (at least one cell)
    int nc = o.n_c > 0 ? o.n_c : std::max(1, (int)floor(1.0 / rc));
    if (1.0 / nc < rc * (1 - 1e-12) && o.n_c <= 0)
        nc = std::max(1, nc - 1);
    if ((double)nc * nc * nc * kSub3 > 2.0e8)
        return EWALD_EUNSUPPORTED;

    p.xi = xi / L;
    p.rc = rc * L;
    p.n_c = nc;
    p.cell = L / nc;
    p.M = M;
    p.h = L / M;
    p.P = P;
    p.est_err = est_near(xi, rc) + est_far(1.0 / M, xi) + est_window(P);
    if (p.near_ds && xi * rc > ERFCX_DS_X)  // beyond the double-single erfcx fit
        p.near_ds = 0;

    // window polynomial degree: max error <= tol/20 (and the FP32 floor)
    double wtarget = std::max(tol / 30.0, p.near_f64 ? 1e-15 : 2e-8);
    int deg = o.poly_deg;
    if (deg <= 0) {
        WindowPoly wp;
        double e = 1.0;
        for (deg = 3; deg <= kMaxDeg; ++deg) {
            if (fit_window(P, deg, &wp, &e) != EWALD_OK)
                return EWALD_EUNSUPPORTED;
            if (e <= wtarget)
                break;
        }
        if (deg > kMaxDeg)
            deg = kMaxDeg;
    }
    p.poly_deg = deg;

    // grid tile T: the FP32 G2P block of (T + P - 1)^3 x 3 values must fit in
    // shared memory (<= 222 KB of the 227 KB a block may use; counted at 16
    // bytes a grid point, above the planar staging's 12); FP64 plans read the
    // grid from L2 in G2P and only need P2G's shared memory, which fits at T = 8
    const double esz = p.near_f64 ? 0.0 : 16.0;
    int T = o.tile > 0 ? o.tile : 8;
    if (T != 4 && T != 8)
        return EWALD_EUNSUPPORTED;
    const double smem_cap = 220.0 * 1024;
    if (pow(T + P - 1, 3) * esz > smem_cap)
        T = 4;
    if (pow(T + P - 1, 3) * esz > smem_cap)
        return EWALD_EUNSUPPORTED;
    if (M % T)
        T = (M % 4 == 0) ? 4 : 0;
    if (T == 0)
        return EWALD_EUNSUPPORTED;
    p.tile = T;

    // P2P work items: warps of <= 32 targets of one cell
    double s = (double)N / ((double)nc * nc * nc);
    (void)s;
    p.p2p_block = 128;  // four independent warps of <= 32 targets each
    // colleague reach K = ceil(rc / cell); the P2P kernel supports K <= 2
    if ((int)ceil(p.rc / p.cell - 1e-12) > 2)
        return EWALD_EUNSUPPORTED;

    // device footprint (bytes) of the plan's workspaces
    int64_t Mh = M / 2 + 1;
    int64_t m3 = (int64_t)M * M * M, mc = (int64_t)M * M * Mh;
    int64_t nkeys = (int64_t)nc * nc * nc * kSub3, ntl = m3 / ((int64_t)T * T * T);
    int64_t fb = 0;
    fb += N * 4 * 6;                                   // keys, slots, perms
    fb += (nkeys + 1) * 8 + (ntl + 1) * 8 + ((int64_t)nc * nc * nc + 1) * 8;
    fb += N * 2 * (p.near_f64 ? 32 : 16) * 2;          // sorted near / tile data
    fb += p.near_ds ? N * 16 : 0;                      // double-single force low parts
    fb += N * 3 * (p.near_f64 ? 8 : 4) * 2;            // un, uf
    fb += 3 * m3 * (p.fft_f64 ? 8 : 4);                // real grid
    fb += 3 * mc * (p.fft_f64 ? 16 : 8);               // half spectrum
    fb += 2 * 3 * m3 * (p.fft_f64 ? 8 : 4);            // cuFFT work areas (estimate)
    if (!p.near_f64 && p.fft_f64)
        fb += 3 * m3 * 4;                              // FP32 copy of the grid for G2P
    if (p.near_ds && grid_ds_supported(P, T, M)) {
        fb += N * 3 * 2 * ds_window_stride(P) * 4;     // double-single window weights
        fb += 2 * 3 * m3 * 4;                          // double-single copy of the grid
    }
    p.footprint_bytes = fb;
    *out = p;
    return EWALD_OK;
}

}  // namespace ewg

extern "C" ewald_status ewald_choose_params(int64_t N, double L, double tol, ewald_dtype dtype,
                                            const ewald_params *ov, ewald_params *out)
{
    return ewg::choose_params(N, L, tol, dtype, ov, out);
}

extern "C" ewald_status ewald_window_eval(int32_t P, int32_t nu, int64_t n, const double *t,
                                          double *w, double *max_err)
{
    if (n < 0 || (n > 0 && (!t || !w)))
        return EWALD_EINVAL;
    ewg::WindowPoly wp;
    double e = 0;
    ewald_status st = ewg::fit_window(P, nu, &wp, &e);
    if (st != EWALD_OK)
        return st;
    int nn = nu + 1;
    for (int64_t i = 0; i < n; ++i) {
        // t in grid units, |t| < P/2: bin l and offset delta with
        // t = l + 1 - P/2 - delta, delta in [0, 1)
        double u = t[i] + 0.5 * P;        // in [0, P)
        if (!(u > 0.0 && u <= (double)P)) {
            w[i] = 0.0;
            continue;
        }
        int l = (int)ceil(u) - 1;         // u in (l, l + 1]
        double delta = (double)(l + 1) - u;
        double z = 2.0 * delta - 1.0;
        double p = 0.0;
        for (int k = nn - 1; k >= 0; --k)
            p = p * z + wp.coef[(size_t)l * nn + k];
        w[i] = p;
    }
    if (max_err)
        *max_err = e;
    return EWALD_OK;
}

extern "C" ewald_status ewald_window_hat(int32_t P, double h, int64_t n, const double *k,
                                         double *what)
{
    if (n < 0 || (n > 0 && (!k || !what)) || P < 2 || P > ewg::kMaxP || !(h > 0))
        return EWALD_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        what[i] = ewg::kb_window_hat(k[i], h, P);
    return EWALD_OK;
}
