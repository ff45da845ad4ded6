"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong constant) fails at
least one of them:

* Hasimoto's cubic-lattice constant fixes the overall constant, the self term
  and the k = 0 convention;
* invariance under the splitting parameter xi ties the near-field kernel of
  eq. (g-near) to the far-field transform of eq. (GFk) term by term;
* symmetry of the mobility operator catches transposed tensor contractions;
* translation invariance catches phase sign errors in the structure factor;
* a brute-force lattice sum of the bare Stokeslet fixes the result itself,
  modulo the affine surface term of a spherical summation order.
"""
import os

import numpy as np
import pytest

from paper_2606_19059_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _xi_sc():
    with open(os.path.join(GOLDEN, "hasimoto_sc.txt")) as fh:
        for line in fh:
            if line.startswith("xi_sc"):
                return float(line.split()[1])
    raise RuntimeError("constant missing")


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L", [1.0, 2.5])
@pytest.mark.parametrize("xi_L", [3.0, 6.0, 10.0])
def test_hasimoto_cubic_lattice(oracle_mod, L, xi_L):
    xi_sc = _xi_sc()
    x = np.array([[0.31, 0.47, 0.52]]) * L
    for f in (np.array([[1.0, 0.0, 0.0]]), np.array([[0.3, -0.5, 0.8]])):
        u = oracle_mod.ewald(x, f, L, xi=xi_L / L)
        expect = -(8.0 / 6.0) * xi_sc * f / L
        assert np.abs(u - expect).max() <= 1e-10 * np.abs(expect).max(), (u, expect)


def test_xi_invariance(oracle_mod):
    x, f = workloads.make("uniform", 24, seed=11)
    us = [oracle_mod.ewald(x, f, 1.0, xi=xi) for xi in (4.0, 7.0, 11.0)]
    for u in us[1:]:
        assert _rel(u, us[0]) < 1e-12


def test_xi_invariance_nonzero_net_force(oracle_mod):
    # the k = 0 mode is dropped, so a net force is allowed; the sum stays xi-free
    rng = np.random.default_rng(5)
    x = rng.random((12, 3)) * 1.7
    f = rng.standard_normal((12, 3)) + 0.5
    u1 = oracle_mod.ewald(x, f, 1.7, xi=3.0)
    u2 = oracle_mod.ewald(x, f, 1.7, xi=8.0)
    assert _rel(u2, u1) < 1e-12


def test_mobility_symmetry(oracle_mod):
    rng = np.random.default_rng(12)
    x = workloads.uniform(rng, 30)
    f, g = workloads.forces(rng, 30), workloads.forces(rng, 30)
    Mf = oracle_mod.ewald(x, f, 1.0)
    Mg = oracle_mod.ewald(x, g, 1.0)
    a, b = np.sum(g * Mf), np.sum(f * Mg)
    assert abs(a - b) <= 1e-12 * np.sqrt(np.sum(Mf**2) * np.sum(g**2))


def test_translation_invariance(oracle_mod):
    x, f = workloads.make("uniform", 25, seed=13)
    shift = np.array([0.377, -0.912, 0.141])
    u1 = oracle_mod.ewald(x, f, 1.0)
    u2 = oracle_mod.ewald(np.mod(x + shift, 1.0), f, 1.0)
    assert _rel(u2, u1) < 1e-12


def test_linearity(oracle_mod):
    rng = np.random.default_rng(14)
    x = workloads.uniform(rng, 16)
    f, g = workloads.forces(rng, 16), workloads.forces(rng, 16)
    u = oracle_mod.ewald(x, 2.0 * f - 3.0 * g, 1.0)
    v = 2.0 * oracle_mod.ewald(x, f, 1.0) - 3.0 * oracle_mod.ewald(x, g, 1.0)
    assert _rel(u, v) < 1e-12


def _affine_residual(ub, ue, x):
    A = np.hstack([np.ones((x.shape[0], 1)), x])
    res = []
    for c in range(3):
        coef, *_ = np.linalg.lstsq(A, ub[:, c] - ue[:, c], rcond=None)
        res.append(ub[:, c] - ue[:, c] - A @ coef)
    return np.abs(np.array(res)).max() / np.abs(ue).max()


def test_brute_force_lattice_sum(oracle_mod):
    # 10 points x 3 components = 30 values against a 12-parameter affine field
    x, f = workloads.make("uniform", 10, seed=15)
    ue = oracle_mod.ewald(x, f, 1.0)
    r20 = _affine_residual(oracle_mod.image_sum(x, f, 1.0, 20.0), ue, x)
    r40 = _affine_residual(oracle_mod.image_sum(x, f, 1.0, 40.0), ue, x)
    assert r40 < 5e-7
    assert r40 < 0.25 * r20  # the residual shrinks with the radius


def test_near_field_small_xi_is_bare_stokeslet(oracle_mod):
    # xi -> 0: G^N -> G (bracket -> 1, diagonal term -> 0), so two points
    # closer than rc feel the bare Stokeslet of Sec. 2
    x = np.array([[0.2, 0.3, 0.4], [0.25, 0.28, 0.47]])
    f = np.array([[0.0, 0.0, 0.0], [0.7, -0.2, 0.4]])
    u = oracle_mod.near_field(x, f, 1.0, xi=1e-9, rc=0.2)
    r = x[0] - x[1]
    rn = np.linalg.norm(r)
    bare = f[1] / rn + r * np.dot(r, f[1]) / rn**3
    assert np.allclose(u[0], bare, rtol=1e-8)


def test_near_field_cutoff_is_inclusive_and_self_term(oracle_mod):
    # one pair at distance exactly 0.125 (exactly representable): kept at
    # rc = 0.125, dropped just below, where only the self term -(4 xi/sqrt pi) f
    # is left; a lone point sees no image (distance 1 > 0.9), only itself
    x = np.array([[0.5, 0.5, 0.5], [0.625, 0.5, 0.5]])
    f = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    self_term = -oracle_mod.self_coefficient(5.0) * f
    u_in = oracle_mod.near_field(x, f, 1.0, xi=5.0, rc=0.125)
    u_out = oracle_mod.near_field(x, f, 1.0, xi=5.0, rc=0.1249)
    assert np.abs(u_in - self_term).max() > 0
    assert np.abs(u_out - self_term).max() == 0
    lone = oracle_mod.near_field(x[:1], f[:1], 1.0, xi=5.0, rc=0.9)
    assert np.abs(lone - self_term[:1]).max() == 0


def test_coincident_points_xi_invariance(oracle_mod):
    # a point duplicated exactly: its pair is skipped as a whole (near and far
    # part), so the sum must not depend on xi
    x, f = workloads.make("uniform", 15, seed=17)
    x[9] = x[4]
    x[12] = x[4]
    us = [oracle_mod.ewald(x, f, 1.0, xi=xi) for xi in (4.0, 9.0)]
    assert _rel(us[1], us[0]) < 1e-12
    # and equals the sum in which the three copies carry one combined force
    # seen by the other points, while each copy ignores the other two
    keep = [i for i in range(15) if i not in (9, 12)]
    g = f.copy()
    g[4] = f[4] + f[9] + f[12]
    u_merged = oracle_mod.ewald(x[keep], g[keep], 1.0, xi=6.0)
    others = [k for k, i in enumerate(keep) if i != 4]
    assert _rel(us[0][[i for i in keep if i != 4]], u_merged[others]) < 1e-12


def test_far_field_box_equals_sphere_when_it_contains_it(oracle_mod):
    x, f = workloads.make("uniform", 8, seed=16)
    xi = 3.0
    # sphere |k| < 2 xi sqrt(40) ~ 37.9 -> |m| <= 6; a box of 8 contains it,
    # and the extra box modes carry e^{-k^2/4xi^2} < e^{-40}
    ub = oracle_mod.far_field(x, f, 1.0, xi, kbox=8)
    us = oracle_mod.far_field(x, f, 1.0, xi, kbox=0)
    assert _rel(ub, us) < 1e-14
