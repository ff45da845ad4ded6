"""Host-side checks of the CUDA library (no GPU needed): it builds, loads and
exports every function of include/ewald_gb300.h; the planner's parameter
choice follows eq. (ese); the plan-time window fit and window transform agree
with the oracle's exact Kaiser-Bessel window; the erf/erfcx fits meet their
stated error bounds."""
import os
import re

import numpy as np
import pytest
from scipy import special

from oracle import spectral
from paper_2606_19059_gb300 import ewald

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ewald_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ewald_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = ewald.load()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ewald.EXPORTED)


def test_status_strings():
    assert ewald.ewald_status_string(0) == "ok"
    assert "invalid" in ewald.ewald_status_string(1)


@pytest.mark.parametrize("M,P,tol,nc_ref", [
    (128, 12, 1e-6, 9),
    (256, 14, 1e-7, 16),
])
def test_params_with_grid_given(M, P, tol, nc_ref):
    ov = ewald.ewald_params()
    ov.M, ov.P = M, P
    p = ewald.ewald_choose_params(100_000, 1.0, tol, ewald.EWALD_F32_BULK, ov)
    assert p.M == M and p.P == P
    # eq. (ese) with each term at tol/10: E^F at equality fixes xi in closed
    # form, E^N fixes rc (bisection), and n_c = floor(1/rc)
    h, t = 1.0 / M, tol / 10
    xi_ref = np.pi / (2 * h * np.sqrt(np.log(4 / (3 * h) * np.sqrt(3.5) / t)))
    assert p.xi == pytest.approx(xi_ref, rel=1e-12)
    xi, rc = p.xi, p.rc
    EN = lambda r: np.sqrt(112 / 9 * xi**4 * r**3) * np.exp(-(xi * r) ** 2)
    assert EN(rc) <= t * 1.0001 and EN(rc * 0.999) > t
    assert p.n_c == nc_ref == int(np.floor(1.0 / rc)) and p.cell >= p.rc


def test_params_scale_with_box():
    ov = ewald.ewald_params()
    ov.M, ov.P = 64, 10
    a = ewald.ewald_choose_params(5000, 1.0, 1e-6, ewald.EWALD_F64, ov)
    b = ewald.ewald_choose_params(5000, 3.0, 1e-6, ewald.EWALD_F64, ov)
    assert b.xi == pytest.approx(a.xi / 3.0, rel=1e-12)
    assert b.rc == pytest.approx(a.rc * 3.0, rel=1e-12)
    assert b.n_c == a.n_c


def test_params_auto_and_precision_switches():
    p = ewald.ewald_choose_params(1000, 1.0, 1e-8, ewald.EWALD_F64)
    assert p.near_f64 == 1 and p.fft_f64 == 1 and 4 <= p.P <= 16 and p.M % 2 == 0
    q = ewald.ewald_choose_params(100_000, 1.0, 1e-6, ewald.EWALD_F32_BULK)
    assert q.near_f64 == 0 and q.fft_f64 == 0
    r = ewald.ewald_choose_params(100_000, 1.0, 2e-7, ewald.EWALD_F32_BULK)
    assert r.near_f64 == 0 and r.near_ds == 0 and r.fft_f64 == 1
    # plain FP32 stops above 1e-7: tol 1e-7 itself takes the double-single kernels
    r7 = ewald.ewald_choose_params(100_000, 1.0, 1e-7, ewald.EWALD_F32_BULK)
    assert r7.near_f64 == 1 and r7.near_ds == 1 and r7.fft_f64 == 1
    s = ewald.ewald_choose_params(100_000, 1.0, 1e-9, ewald.EWALD_F32_BULK)
    assert s.near_f64 == 1  # FP32 cannot reach 1e-9
    assert 0 < p.est_err <= 1e-8 and 0 < q.est_err <= 1e-6


@pytest.mark.parametrize("N,L,tol,status", [
    (0, 1.0, 1e-6, ewald.EWALD_EINVAL),
    (10, -1.0, 1e-6, ewald.EWALD_EINVAL),
    (10, 1.0, 0.5, ewald.EWALD_EINVAL),
    (10, 1.0, 1e-13, ewald.EWALD_EINVAL),
    (10, float("nan"), 1e-6, ewald.EWALD_EINVAL),
])
def test_params_reject_bad_arguments(N, L, tol, status):
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_choose_params(N, L, tol)
    assert e.value.status == status


def test_params_reject_unsupported_override():
    ov = ewald.ewald_params()
    ov.P = 17
    with pytest.raises(ewald.EwaldError) as e:
        ewald.ewald_choose_params(100, 1.0, 1e-6, ewald.EWALD_F64, ov)
    assert e.value.status == ewald.EWALD_EUNSUPPORTED


@pytest.mark.parametrize("P,nu", [(6, 6), (12, 10), (14, 12), (13, 9), (16, 14)])
def test_window_polynomial_fit_matches_exact_window(P, nu):
    t = np.linspace(-P / 2 + 1e-9, P / 2 - 1e-9, 4001)
    w, maxerr = ewald.ewald_window_eval(P, nu, t)
    exact = spectral.kb_window(t, P, 1.0)  # h = 1: t in grid units
    err = np.abs(w - exact).max()
    assert err <= 1.05 * maxerr + 1e-15
    assert maxerr < 1e-3
    assert w[len(t) // 2] == pytest.approx(1.0, abs=maxerr + 1e-15)


def test_window_fit_error_drops_with_degree():
    errs = [ewald.ewald_window_eval(12, nu, np.zeros(1))[1] for nu in (4, 6, 8, 10)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-10


def test_planner_degree_meets_tolerance():
    for tol, dt in ((1e-6, ewald.EWALD_F32_BULK), (1e-8, ewald.EWALD_F64), (1e-10, ewald.EWALD_F64)):
        ov = ewald.ewald_params()
        ov.M, ov.P = 64, 12
        p = ewald.ewald_choose_params(1000, 1.0, tol, dt, ov)
        _, e = ewald.ewald_window_eval(p.P, p.poly_deg, np.zeros(1))
        assert e <= max(tol / 20, 2e-8 if p.near_f64 == 0 else 1e-15) * 1.0001


@pytest.mark.parametrize("P", [4, 9, 12, 16])
def test_window_transform_matches_oracle(P):
    h = 1.0 / 48
    beta, aw = spectral.kb_params(P, h)
    k = np.linspace(0.0, 3.0 * beta / aw, 301)
    ours = ewald.ewald_window_hat(P, h, k)
    ref = spectral.kb_window_hat(k, P, h)
    assert np.abs(ours - ref).max() <= 1e-12 * abs(ref[0])


def _read_header_coeffs():
    src = open(os.path.join(ROOT, "paper_2606_19059_gb300", "csrc", "erf_rational.h")).read()

    def arr(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])

    def const(name):
        return float(re.search(r"#define " + name + r" ([0-9.eE+-]+)", src).group(1))

    return arr("erf_rat_f64_p"), arr("erf_rat_f64_q"), arr("erfcx_f32_c"), const


def test_erf_rational_fp64_meets_bound():
    p, q, _, const = _read_header_coeffs()
    X = const("ERF_RAT_X64")
    x = np.linspace(1e-6, X, 50001)
    z = 2 * x / X - 1
    r = np.polyval(p[::-1], z) / np.polyval(q[::-1], z)
    err = np.abs(r - special.erf(x) / x).max()
    # Horner in double: the bound the kernel meets (exact-arithmetic error is smaller)
    assert err <= 1.5 * const("ERF_RAT_F64_MAXERR_EVAL") + 1e-15
    assert const("ERF_RAT_F64_MAXERR") < 1e-12 and err < 1e-11


def test_erfcx_fp32_form_meets_bound():
    _, _, c, const = _read_header_coeffs()
    X, C = const("ERFCX_X32"), const("ERFCX_C32")
    x = np.linspace(0.0, X, 50001)
    t = 1.0 / (1.0 + C * x)
    g = t * np.polyval(c[::-1], t)
    rel = np.abs(g - special.erfcx(x)) / special.erfcx(x)
    assert rel.max() <= 1.5 * const("ERFCX_F32_MAXERR")
    assert rel.max() < 1e-8


def test_apply_entry_points_reject_null_plan_on_the_host():
    # argument checks come before any CUDA call, so they run without a GPU
    for fn, nargs in ((ewald.ewald_apply, 3), (ewald.ewald_apply_forces, 2),
                      (ewald.ewald_apply_combined, 5), (ewald.ewald_apply_host, 3)):
        with pytest.raises(ewald.EwaldError) as e:
            fn(None, *([None] * nargs))
        assert e.value.status == ewald.EWALD_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the CUDA library the binding raises
    monkeypatch.setattr(ewald, "_lib", None)
    monkeypatch.setattr(ewald, "LIB_PATH", str(tmp_path / "libewald_gb300.so"))
    with pytest.raises(RuntimeError, match="CUDA library not built"):
        ewald.load(build_if_missing=False)
