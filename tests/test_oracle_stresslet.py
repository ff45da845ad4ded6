"""Pins of the double-layer (stresslet) oracle, Sec. 2.3, against facts fixed
independently of its own formulas:

* the periodic sum does not depend on the splitting parameter xi (a wrong
  T^N or T-hat^F term breaks the cancellation between the two parts);
* close points in a large box see the bare stresslet -6 r r r / r^5 (pins
  the overall sign and scale, which xi-independence cannot);
* with D = I at every source the double layer is 6 grad of the periodic
  Coulomb potential (T_jll = -6 r_j / r^3), computed by a separate textbook
  Ewald routine that is itself pinned by the rock-salt Madelung constant;
* T is odd in r and symmetric in its last two indices;
* the grid pipeline (spread, FFT, CNV, IFFT, gather) reproduces the direct
  k sum of the far part.
"""
import os

import numpy as np
import pytest

from oracle import stresslet as dl
from paper_2606_19059_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_D(rng, n):
    return dl.densities(rng.standard_normal((n, 3)), rng.standard_normal((n, 3)))


def test_sum_is_independent_of_xi():
    rng = np.random.default_rng(301)
    x = workloads.uniform(rng, 20, 1.0)
    D = _random_D(rng, 20)
    a = dl.ewald(x, D, 1.0, xi=3.0)
    b = dl.ewald(x, D, 1.0, xi=5.5)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_nonunit_box_is_independent_of_xi():
    rng = np.random.default_rng(302)
    L = 2.5
    x = workloads.uniform(rng, 12, L)
    D = _random_D(rng, 12)
    a = dl.ewald(x, D, L, xi=3.0 / L)
    b = dl.ewald(x, D, L, xi=5.0 / L)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_close_points_see_the_bare_stresslet():
    rng = np.random.default_rng(303)
    x = 0.5 + 1e-3 * rng.standard_normal((4, 3))
    D = _random_D(rng, 4)
    u = dl.ewald(x, D, 1.0, xi=4.0)
    free = np.zeros_like(u)
    for i in range(4):
        for j in range(4):
            if i != j:
                free[i] += dl.apply_free(x[i] - x[j], D[j])
    # image and zero-mode corrections are O(|D| / L^2), the pair terms
    # O(|D| / (1e-3)^2)
    assert np.abs(u - free).max() <= 1e-4 * np.abs(free).max()


def _madelung():
    with open(os.path.join(GOLDEN, "madelung_rock_salt.txt")) as fh:
        for line in fh:
            if line.startswith("alpha"):
                return float(line.split()[1])
    raise AssertionError("no alpha line")


@pytest.mark.parametrize("xi", [3.0, 6.0])
def test_coulomb_ewald_gives_the_rock_salt_madelung_constant(xi):
    na = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    cl = np.array([[.5, 0, 0], [0, .5, 0], [0, 0, .5], [.5, .5, .5]], dtype=np.float64)
    y = np.vstack([na, cl])
    c = np.array([1.0] * 4 + [-1.0] * 4)
    phi = dl.coulomb_site_potential(y, c, 1.0, xi)
    r0 = 0.5
    np.testing.assert_allclose(phi[:4], -_madelung() / r0, rtol=1e-12)
    np.testing.assert_allclose(phi[4:], _madelung() / r0, rtol=1e-12)


def test_identity_density_is_six_times_the_coulomb_field():
    rng = np.random.default_rng(304)
    ns, nt = 10, 5
    y = workloads.uniform(rng, ns, 1.0)
    xt = workloads.uniform(rng, nt, 1.0)
    # targets at least 0.1 from every source image (finite differences below)
    d = xt[:, None, :] - y[None, :, :]
    d -= np.rint(d)
    keep = np.sqrt((d * d).sum(-1)).min(1) > 0.1
    xt = xt[keep]
    x = np.vstack([y, xt])
    D = np.zeros((x.shape[0], 3, 3))
    D[:ns] = np.eye(3)
    tid = np.arange(ns, x.shape[0])
    u = dl.ewald(x, D, 1.0, xi=4.0, targets=tid)
    h = 1e-5
    grad = np.zeros_like(u)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        grad[:, a] = (dl.coulomb_potential(xt + e, y, np.ones(ns), 1.0, 4.0)
                      - dl.coulomb_potential(xt - e, y, np.ones(ns), 1.0, 4.0)) / (2 * h)
    assert np.abs(u - 6.0 * grad).max() <= 1e-6 * np.abs(u).max()


def test_kernel_is_odd():
    rng = np.random.default_rng(305)
    x = workloads.uniform(rng, 2, 1.0)
    D = _random_D(rng, 1)
    Da = np.zeros((2, 3, 3))
    Da[1] = D[0]
    Db = np.zeros((2, 3, 3))
    Db[0] = D[0]
    ua = dl.ewald(x, Da, 1.0, xi=4.0, targets=[0])   # source at x1, target x0
    ub = dl.ewald(x, Db, 1.0, xi=4.0, targets=[1])   # source at x0, target x1
    np.testing.assert_allclose(ua, -ub, rtol=1e-10, atol=1e-12 * np.abs(ua).max())


def test_only_the_symmetric_part_of_q_n_enters():
    rng = np.random.default_rng(306)
    x = workloads.uniform(rng, 15, 1.0)
    q, n = rng.standard_normal((15, 3)), rng.standard_normal((15, 3))
    a = dl.ewald(x, dl.densities(q, n), 1.0, xi=4.0)
    b = dl.ewald(x, dl.densities(n, q), 1.0, xi=4.0)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(a).max())
    # an antisymmetric density gives nothing
    A = dl.densities(q, n) - dl.densities(n, q)
    z = dl.ewald(x, A, 1.0, xi=4.0)
    assert np.abs(z).max() <= 1e-12 * np.abs(a).max()


def test_near_field_is_the_real_space_part():
    rng = np.random.default_rng(307)
    x = workloads.uniform(rng, 25, 1.0)
    D = _random_D(rng, 25)
    xi = 5.0
    un = dl.near_field(x, D, 1.0, xi, 6.5 / xi)
    uf = dl.far_field(x, D, 1.0, xi)
    np.testing.assert_allclose(un + uf, dl.ewald(x, D, 1.0, xi=xi), rtol=1e-13, atol=0)
    # a cutoff keeps only pairs within it: compare with the pairwise sum
    rc = 0.2
    uc = dl.near_field(x, D, 1.0, xi, rc)
    ref = np.zeros_like(uc)
    for i in range(25):
        for j in range(25):
            r = x[i] - x[j]
            r -= np.rint(r)
            rr = np.sqrt(r @ r)
            if 0 < rr <= rc:
                ref[i] += dl.apply_near(r, D[j], xi)
    np.testing.assert_allclose(uc, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_grid_pipeline_matches_direct_k_sum():
    rng = np.random.default_rng(308)
    x = workloads.uniform(rng, 24, 1.0)
    D = _random_D(rng, 24)
    M, xi = 32, 8.0
    ud = dl.far_field(x, D, 1.0, xi, kbox=M // 2 - 1)
    errs = {}
    for P in (6, 9, 12):
        us = dl.far_field_spectral(x, D, 1.0, M, P, xi)
        errs[P] = np.abs(us - ud).max() / np.abs(ud).max()
    assert errs[12] < 1e-9
    assert errs[6] > errs[9] > errs[12]
