"""Pins of the numpy far-field reference (oracle/spectral.py), no GPU.

* the closed-form window transform against numerical quadrature of the window;
* P2G and G2P are adjoint (h^3 <P2G f, v> = <f, G2P v>) -- catches a
  transposed or mirrored index between the two stages;
* spreading conserves the total force up to the window's aliasing error;
* the whole spectral far field equals the direct k-space sum of the C oracle
  over the grid's k set, to the window's error (Sec. 2.2, eq. (sca));
* that error shrinks as the support P grows (E^w of eq. (ese)).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import spectral
from paper_2606_19059_gb300 import workloads


@pytest.mark.parametrize("P", [6, 12, 14])
@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_window_transform_closed_form(P):
    h = 1.0 / 32
    beta, aw = spectral.kb_params(P, h)
    for ka in (0.0, 0.3 * beta, 0.999 * beta, beta, 1.4 * beta, 2.5 * beta):
        k = ka / aw
        num, _ = integrate.quad(lambda t: spectral.kb_window(t, P, h) * np.cos(k * t),
                                -aw, aw, limit=400, epsabs=1e-16, epsrel=1e-13)
        closed = spectral.kb_window_hat(np.array([k]), P, h)[0]
        scale = spectral.kb_window_hat(np.array([0.0]), P, h)[0]
        assert abs(num - closed) <= 1e-11 * scale, (P, ka, num, closed)


def test_window_shape():
    h = 0.1
    P = 8
    _, aw = spectral.kb_params(P, h)
    t = np.linspace(-aw, aw, 101)
    w = spectral.kb_window(t, P, h)
    assert w[50] == pytest.approx(1.0)          # w_0(0) = I0(beta)/I0(beta)
    assert np.allclose(w, w[::-1])              # even
    assert w[0] == 0.0 and w[-1] == 0.0         # truncated at |t| = a_w
    assert np.all(np.diff(w[:51]) > 0)          # increasing towards the centre


def test_spread_gather_adjoint():
    rng = np.random.default_rng(21)
    L, M, P = 1.3, 16, 7
    x = workloads.uniform(rng, 9, L)
    f = workloads.forces(rng, 9, zero_mean=False)
    v = rng.standard_normal((3, M, M, M))
    h = L / M
    lhs = h ** 3 * np.sum(spectral.spread(x, f, L, M, P) * v)
    rhs = np.sum(f * spectral.gather(x, v, L, M, P))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_spread_conserves_force():
    rng = np.random.default_rng(22)
    L, M, P = 1.0, 24, 12
    x = workloads.uniform(rng, 7, L)
    f = workloads.forces(rng, 7, zero_mean=False)
    phi = spectral.spread(x, f, L, M, P)
    h = L / M
    w0 = spectral.kb_window_hat(np.array([0.0]), P, h)[0]
    total = h ** 3 * phi.reshape(3, -1).sum(axis=1)
    assert np.allclose(total, w0 ** 3 * f.sum(axis=0), rtol=1e-9, atol=1e-9 * np.abs(f).sum())


def test_spread_wraps_support_larger_than_grid():
    # P > M: the window wraps onto itself; the force is still conserved
    L, M, P = 1.0, 6, 9
    x = np.array([[0.05, 0.93, 0.5]])
    f = np.array([[1.0, -2.0, 0.5]])
    phi = spectral.spread(x, f, L, M, P)
    h = L / M
    w0 = spectral.kb_window_hat(np.array([0.0]), P, h)[0]
    assert np.allclose(h ** 3 * phi.reshape(3, -1).sum(axis=1), w0 ** 3 * f[0], rtol=1e-5)


def test_far_field_matches_direct_k_sum(oracle_mod):
    x, f = workloads.make("uniform", 30, seed=23)
    M, xi = 32, 8.0
    ud = oracle_mod.far_field(x, f, 1.0, xi, kbox=M // 2 - 1)
    errs = {}
    for P in (6, 9, 12):
        us = spectral.far_field(x, f, 1.0, M, P, xi)
        errs[P] = np.abs(us - ud).max() / np.abs(ud).max()
    assert errs[12] < 1e-10
    assert errs[6] > errs[9] > errs[12]


def test_far_field_nonunit_box(oracle_mod):
    L = 2.0
    rng = np.random.default_rng(24)
    x = workloads.uniform(rng, 12, L)
    f = workloads.forces(rng, 12)
    M, P, xi = 24, 12, 4.0 / L
    ud = oracle_mod.far_field(x, f, L, xi, kbox=M // 2 - 1)
    us = spectral.far_field(x, f, L, M, P, xi)
    assert np.abs(us - ud).max() <= 1e-10 * np.abs(ud).max()
