"""Fit the rational approximants used by the near-field (P2P) kernel and write
``csrc/erf_rational.h``.

Sec. 4 of the paper replaces the library erf/erfc in the near-field kernel by
a rational approximant of erf(x)/x evaluated with FMAs and one division, and
forms erfc(x)/x = 1/x - erf(x)/x.  Two approximants are built here, each with
its own coefficients:

* FP64 kernel -- the paper's form: erf(x)/x ~= P(z)/Q(z), degrees 13/13, in the
  centred variable z = 2x/X64 - 1 on x in [0, X64] (centring keeps the
  monomial coefficients moderate).  Fitted by the Sanathanan-Koerner
  linearised least-squares iteration followed by Lawson reweighting towards
  the minimax error, in 50-digit mpmath arithmetic.

* FP32 kernel -- in single precision the rational P/Q cancels inside its own
  sums (its denominator is small where its coefficients are large); measured,
  it loses about 1e-5 in Horner or Clenshaw form.  The FP32 kernel splits at
  x = 1:
    x < 1:  the paper's form erfc(x)/x = 1/x - erf(x)/x with erf(x)/x a
            degree-8 polynomial in x^2 (well conditioned there), so the
            dominant 1/r of a close pair is not touched by any approximation;
    x >= 1: erfcx(x) = e^{x^2} erfc(x) ~= t p(t), t = 1/(1 + x/2) (the
            Chebyshev-type substitution of Numerical Recipes' erfcc), degree 9,
            fitted for minimax *relative* error, times the e^{-x^2} the kernel
            evaluates anyway for the Gaussian term of eq. (g-near); no
            cancellation, and erfc(1) = 0.16 damps the exponential's error.
  Still FMAs and one division per pair.

Each fit's maximum error on a dense grid against 50-digit erf is written
beside the coefficients and re-checked by the test suite.

Run:  python -m paper_2606_19059_gb300.fit_erf
"""
from __future__ import annotations

import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50
X64 = 7.0           # FP64 interval: xi * rc <= 7 covers tol down to 1e-12
X32 = 6.0           # FP32 interval (the paper's [0, 6])
C32 = 0.5           # t = 1 / (1 + C32 x)
DEG32 = 9
DEG64 = 13
XS32 = 1.0          # FP32 small-x branch: erf(x)/x as a polynomial in x^2 on [0, XS32]
DEGS32 = 8
DEGX2 = 6           # FP32 2^f on [-1/2, 1/2] (tight-tolerance exponential)
# Double-single (pairs of FP32) near field, tol down to 1e-9: erfcx(x) = t g(u)
# on x in [0, XDS], t = 1 / (1 + x/2) in [1/4, 1], u = (8 t - 5) / 3 in [-1, 1],
# g a degree-DEGDS polynomial (Chebyshev interpolation, monomial form); terms
# below DSSPLIT carry two-float coefficients, the rest one float.
XDS = 6.0
DEGDS = 16
DSSPLIT = 9
EXPDS_N = 13        # e^s, |s| <= ln2 / 2: Taylor terms 0..13; two-float for 3..5


def erf_over_x(x):
    x = mp.mpf(x)
    if x == 0:
        return 2 / mp.sqrt(mp.pi)
    return mp.erf(x) / x


def erfcx(x):
    x = mp.mpf(x)
    return mp.erfc(x) * mp.exp(x * x)


def _horner(c, t):
    s = mp.mpf(0)
    for a in reversed(c):
        s = s * t + a
    return s


def fit_rational_erf_over_x(n_p: int, n_q: int, n_pts: int = 300, sk_iters: int = 10,
                            lawson_iters: int = 40):
    """P, Q (lowest degree first, Q[0] = 1) with P(z)/Q(z) ~ erf(x)/x,
    z = 2x/X64 - 1."""
    zs = [-mp.cos(mp.pi * (i + mp.mpf(0.5)) / n_pts) for i in range(n_pts)]
    gs = [erf_over_x((z + 1) * X64 / 2) for z in zs]
    q = [mp.mpf(1)] + [mp.mpf(0)] * n_q
    w = [mp.mpf(1)] * n_pts
    p = None
    for it in range(sk_iters + lawson_iters):
        rows, rhs = [], []
        for z, g, wi in zip(zs, gs, w):
            s = mp.sqrt(wi) / _horner(q, z)
            rows.append([s * z ** k for k in range(n_p + 1)] +
                        [-s * g * z ** k for k in range(1, n_q + 1)])
            rhs.append(s * g)
        A, b = mp.matrix(rows), mp.matrix(rhs)
        sol = mp.lu_solve(A.T * A, A.T * b)
        p = [sol[k] for k in range(n_p + 1)]
        q = [mp.mpf(1)] + [sol[n_p + 1 + k] for k in range(n_q)]
        if it >= sk_iters:
            err = [abs(_horner(p, z) / _horner(q, z) - g) for z, g in zip(zs, gs)]
            tot = mp.fsum(wi * e for wi, e in zip(w, err))
            w = [wi * e / tot * n_pts for wi, e in zip(w, err)]
    return p, q


def fit_erfcx(deg: int, n_pts: int = 3001, iters: int = 80):
    """c[0..deg] with erfcx(x) ~= t * sum_k c[k] t^k, t = 1/(1 + C32 x)."""
    x = np.linspace(0.0, X32, n_pts)
    g = np.array([float(erfcx(v)) for v in x])
    t = 1.0 / (1.0 + C32 * x)
    V = np.vstack([t ** (k + 1) for k in range(deg + 1)]).T
    w = np.ones_like(x)
    coef = None
    for _ in range(iters):
        W = np.sqrt(w) / g
        coef, *_ = np.linalg.lstsq(V * W[:, None], g * W, rcond=None)
        e = np.abs(V @ coef - g) / g
        w = w * e
        w /= w.mean()
    return [float(c) for c in coef]


def fit_erfx_small(deg: int, n_pts: int = 2001, iters: int = 60):
    """a[0..deg] with erf(x)/x ~= sum_k a[k] (x^2)^k on [0, XS32] (minimax
    absolute error by Lawson reweighting)."""
    x = np.linspace(0.0, XS32, n_pts)
    g = np.array([float(erf_over_x(v)) for v in x])
    t = x * x
    V = np.vstack([t ** k for k in range(deg + 1)]).T
    w = np.ones_like(x)
    coef = None
    for _ in range(iters):
        W = np.sqrt(w)
        coef, *_ = np.linalg.lstsq(V * W[:, None], g * W, rcond=None)
        e = np.abs(V @ coef - g)
        w = w * e
        w /= w.mean()
    return [float(c) for c in coef]


def max_error_small(a, n_check: int = 20001) -> float:
    """max |sum a_k x^{2k} - erf(x)/x| on [0, XS32] (exact arithmetic)."""
    m = mp.mpf(0)
    for i in range(n_check):
        x = XS32 * mp.mpf(i) / (n_check - 1)
        m = max(m, abs(_horner(a, x * x) - erf_over_x(x)))
    return float(m)


def fit_exp2(deg: int, n_pts: int = 2001, iters: int = 60):
    """c[0..deg] with 2^f ~= sum_k c[k] f^k on [-1/2, 1/2], minimax relative
    error (Lawson reweighting); used by the tight-tolerance FP32 kernel to
    evaluate e^{-x^2} = 2^(n + f) without the hardware approximation."""
    f = np.linspace(-0.5, 0.5, n_pts)
    g = np.array([float(mp.power(2, mp.mpf(v))) for v in f])
    V = np.vstack([f ** k for k in range(deg + 1)]).T
    w = np.ones_like(f)
    coef = None
    for _ in range(iters):
        W = np.sqrt(w) / g
        coef, *_ = np.linalg.lstsq(V * W[:, None], g * W, rcond=None)
        e = np.abs(V @ coef - g) / g
        w = w * e
        w /= w.mean()
    return [float(c) for c in coef]


def max_rel_error_exp2(c, n_check: int = 20001) -> float:
    m = mp.mpf(0)
    for i in range(n_check):
        f = mp.mpf(-0.5) + mp.mpf(i) / (n_check - 1)
        m = max(m, abs(_horner(c, f) / mp.power(2, f) - 1))
    return float(m)


def max_error_f64(p, q, n_check: int = 20001) -> float:
    """max |P(z)/Q(z) - erf(x)/x| on a uniform grid of x in [0, X64]."""
    m = mp.mpf(0)
    for i in range(n_check):
        z = 2 * mp.mpf(i) / (n_check - 1) - 1
        m = max(m, abs(_horner(p, z) / _horner(q, z) - erf_over_x((z + 1) * X64 / 2)))
    return float(m)


def max_error_f64_evaluated(p, q, n_check: int = 20001) -> float:
    """The same error with P and Q evaluated by Horner in IEEE double (the
    kernel's arithmetic): the monomial sums cancel, so this is the bound that
    holds in practice."""
    pf = np.array([float(c) for c in p])
    qf = np.array([float(c) for c in q])
    x = np.linspace(0.0, X64, n_check)
    z = 2.0 * x / X64 - 1.0
    P = np.zeros_like(z)
    Q = np.zeros_like(z)
    for c in pf[::-1]:
        P = P * z + c
    for c in qf[::-1]:
        Q = Q * z + c
    ref = np.array([float(erf_over_x(v)) for v in x])
    return float(np.abs(P / Q - ref).max())


def max_rel_error_f32(c, n_check: int = 20001) -> float:
    """max |t p(t) - erfcx(x)| / erfcx(x) on [0, X32] (exact arithmetic)."""
    m = mp.mpf(0)
    for i in range(n_check):
        x = X32 * mp.mpf(i) / (n_check - 1)
        t = 1 / (1 + C32 * x)
        m = max(m, abs(t * _horner(c, t) - erfcx(x)) / erfcx(x))
    return float(m)


def _g_ds(u):
    t = (3 * mp.mpf(u) + 5) / 8
    x = (1 / t - 1) * 2
    return erfcx(x) / t


def fit_erfcx_ds(deg: int):
    """Monomial coefficients in u of the degree-`deg` Chebyshev interpolant of g."""
    nodes = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (deg + 1)) for k in range(deg + 1)]
    V = mp.matrix([[u ** j for j in range(deg + 1)] for u in nodes])
    c = mp.lu_solve(V, mp.matrix([_g_ds(u) for u in nodes]))
    return [c[i] for i in range(deg + 1)]


def max_rel_error_ds(c, n_check: int = 4001) -> float:
    """max |t g(u) - erfcx(x)| / erfcx(x) over x in [0, XDS] (exact arithmetic,
    coefficients as stored: two floats below DSSPLIT, one float above)."""
    cs = []
    for k, v in enumerate(c):
        hi = float(np.float32(float(v)))
        lo = float(np.float32(float(v - hi))) if k < DSSPLIT else 0.0
        cs.append(mp.mpf(hi) + mp.mpf(lo))
    m = mp.mpf(0)
    for i in range(n_check):
        u = -1 + 2 * mp.mpf(i) / (n_check - 1)
        m = max(m, abs(_horner(cs, u) - _g_ds(u)) / _g_ds(u))
    return float(m)


def two_float(v):
    hi = np.float32(float(v))
    lo = np.float32(float(mp.mpf(v) - mp.mpf(float(hi))))
    return float(hi), float(lo)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out = os.path.join(here, "csrc", "erf_rational.h")
    p, q = fit_rational_erf_over_x(DEG64, DEG64)
    e64 = max_error_f64(p, q)
    e64e = max_error_f64_evaluated(p, q)
    c32 = fit_erfcx(DEG32)
    e32 = max_rel_error_f32(c32)
    s32 = fit_erfx_small(DEGS32)
    es32 = max_error_small(s32)
    print("f32 erf(x)/x small-x poly", DEGS32, "max abs error", es32)
    x2 = fit_exp2(DEGX2)
    ex2 = max_rel_error_exp2(x2)
    print("f32 2^f poly", DEGX2, "max rel error", ex2)
    cds = fit_erfcx_ds(DEGDS)
    eds = max_rel_error_ds(cds)
    print("double-single erfcx g(u)", DEGDS, "max rel error", eds)
    print("f64 erf(x)/x  P/Q", DEG64, "max abs error", e64)
    print("f32 erfcx  t p(t)", DEG32, "max rel error", e32)
    L = [
        "/* Generated by paper_2606_19059_gb300/fit_erf.py -- do not edit.",
        " *",
        " * FP64: erf(x)/x ~= P(z)/Q(z), z = 2x/ERF_RAT_X64 - 1, 0 <= x <= ERF_RAT_X64",
        " *       (Sec. 4: rational approximation of erf(x)/x, FMAs + one division).",
        " * FP32: erfcx(x) = e^{x^2} erfc(x) ~= t p(t), t = 1/(1 + ERFCX_C32 x),",
        " *       0 <= x <= ERFCX_X32.",
        " * Coefficients lowest degree first; *_MAXERR measured against 50-digit erf.",
        " */",
        "#pragma once",
        "",
        f"#define ERF_RAT_X64 {X64!r}",
        f"#define ERF_RAT_F64_N {DEG64 + 1}",
        f"#define ERF_RAT_F64_MAXERR {e64:.3e}  /* absolute, on erf(x)/x, exact arithmetic */",
        f"#define ERF_RAT_F64_MAXERR_EVAL {e64e:.3e}  /* same, Horner in IEEE double */",
        f"static const double erf_rat_f64_p[{DEG64 + 1}] = {{",
    ]
    L += [f"    {mp.nstr(v, 21, min_fixed=-1, max_fixed=-1)}," for v in p]
    L += ["};", f"static const double erf_rat_f64_q[{DEG64 + 1}] = {{"]
    L += [f"    {mp.nstr(v, 21, min_fixed=-1, max_fixed=-1)}," for v in q]
    L += ["};", "",
          f"#define ERFCX_X32 {X32!r}",
          f"#define ERFCX_C32 {C32!r}",
          f"#define ERFCX_F32_N {DEG32 + 1}",
          f"#define ERFCX_F32_MAXERR {e32:.3e}  /* relative, on erfcx(x) */",
          f"static const double erfcx_f32_c[{DEG32 + 1}] = {{"]
    L += [f"    {v!r}," for v in c32]
    L += ["};", "",
          f"#define ERFX_SMALL_X32 {XS32!r}",
          f"#define ERFX_SMALL_N {DEGS32 + 1}",
          f"#define ERFX_SMALL_MAXERR {es32:.3e}  /* absolute, on erf(x)/x */",
          f"static const double erfx_small_c[{DEGS32 + 1}] = {{"]
    L += [f"    {v!r}," for v in s32]
    L += ["};", "",
          f"#define EXP2_F32_N {DEGX2 + 1}",
          f"#define EXP2_F32_MAXERR {ex2:.3e}  /* relative, on 2^f, |f| <= 1/2 */",
          f"static const double exp2_f32_c[{DEGX2 + 1}] = {{"]
    L += [f"    {v!r}," for v in x2]
    L += ["};", "",
          "/* Double-single near field: erfcx(x) = t g(u), t = 1/(1 + x/2), u = (8t - 5)/3,",
          " * x in [0, ERFCX_DS_X]; g_k = hi + lo for k < ERFCX_DS_SPLIT, hi alone above. */",
          f"#define ERFCX_DS_X {XDS!r}",
          f"#define ERFCX_DS_N {DEGDS + 1}",
          f"#define ERFCX_DS_SPLIT {DSSPLIT}",
          f"#define ERFCX_DS_MAXERR {eds:.3e}  /* relative, on erfcx(x), coefficients as stored */",
          f"static const float erfcx_ds_hi[{DEGDS + 1}] = {{"]
    L += [f"    {two_float(v)[0]!r}f," for v in cds]
    L += ["};", f"static const float erfcx_ds_lo[{DSSPLIT}] = {{"]
    L += [f"    {two_float(v)[1]!r}f," for v in cds[:DSSPLIT]]
    L += ["};", "",
          "/* e^s for |s| <= ln2/2: Taylor coefficients 1/k!, k = 0..EXP_DS_N - 1; two floats",
          " * (hi, lo) for the inexact ones among k <= 5. */",
          f"#define EXP_DS_N {EXPDS_N + 1}",
          f"static const float exp_ds_hi[{EXPDS_N + 1}] = {{"]
    L += [f"    {two_float(1 / mp.factorial(k))[0]!r}f," for k in range(EXPDS_N + 1)]
    L += ["};", "static const float exp_ds_lo[6] = {"]
    L += [f"    {two_float(1 / mp.factorial(k))[1]!r}f," for k in range(6)]
    L += ["};", ""]
    with open(out, "w") as fh:
        fh.write("\n".join(L))
    print("wrote", out)


if __name__ == "__main__":
    main()
