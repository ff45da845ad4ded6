"""Host checks (no GPU) of the double-layer near field's FP32 arithmetic:

* positions are cell-local in cell units, q = x / cell - c, split into FP32
  hi (on a 2^-20 lattice) and lo = q - hi;
* the FP32 distance filter on the hi parts, with its threshold grown to
  (rc / cell)(1 + 1e-4) + 1e-5, keeps every pair whose exact distance is <= rc;
* the FP32 separation r = (((t_hi - o) - s_hi) + (t_lo - s_lo)) * cell (o the
  neighbour cell offset; the hi terms are exact) is accurate to a few 1e-7 of
  |r| down to near-coincident points, across cell faces in either direction.

The kernel's FP32 operations are restated with numpy float32 (an FMA rounds
once: the product of two float32 values is exact in float64).
"""
import numpy as np
import pytest

f32 = np.float32


def fmaf(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def split(q):
    X = np.rint(q * 1048576.0) / 1048576.0
    return X.astype(f32), (q - X).astype(f32)


def _pairs(rng, n, cell, rc, L, shell):
    """Targets anywhere in the box, sources at distance rc (1 + shell u),
    u uniform in [-1, 1], in random directions (periodic wrap)."""
    t = rng.random((n, 3)) * L
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rc * (1.0 + shell * rng.uniform(-1.0, 1.0, n))
    s = t - d * r[:, None]
    s -= L * np.floor(s / L)
    return t, s


def _local(v, cell, nc):
    inv = 1.0 / cell
    c = np.clip((v * inv).astype(np.int64), 0, nc - 1)
    return c, v * inv - c


@pytest.mark.parametrize("L,nc,rc_frac", [(1.0, 9, 0.972), (1.0, 16, 0.99), (2.5, 5, 0.6), (1.0, 3, 1.0)])
def test_fp32_filter_keeps_every_pair_within_rc(L, nc, rc_frac):
    rng = np.random.default_rng(11)
    cell = L / nc
    rc = rc_frac * cell
    t, s = _pairs(rng, 200_000, cell, rc, L, 2e-4)
    ct, tl = _local(t, cell, nc)
    cs, sl = _local(s, cell, nc)
    # the neighbour offset o of the source's cell, image included
    o = cs - ct
    o -= nc * np.rint(o / nc).astype(np.int64)
    th, _ = split(tl)
    sh, _ = split(sl)
    b = (th - o.astype(f32)).astype(f32)
    r = (b - sh).astype(f32)
    r2 = fmaf(r[:, 0], r[:, 0], fmaf(r[:, 1], r[:, 1], (r[:, 2] * r[:, 2]).astype(f32)))
    rcm = (rc / cell) * (1.0 + 1e-4) + 1e-5
    passed = r2 <= f32(rcm * rcm)
    # exact separation of the nearest image
    d = t - s
    d -= L * np.rint(d / L)
    exact_in = np.sqrt((d * d).sum(1)) <= rc
    assert exact_in.sum() > 50_000
    assert np.all(passed[exact_in])
    # and the margin is small: few pairs beyond rc (1 + 2e-4) pass
    far = np.sqrt((d * d).sum(1)) > rc * (1 + 2e-4)
    assert not np.any(passed & far)


def test_fp32_separation_from_hi_lo_parts_is_accurate():
    rng = np.random.default_rng(12)
    L, nc = 1.0, 9
    cell = L / nc
    n = 100_000
    t = rng.random((n, 3)) * L
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # separations from 1e-6 cell to one cell, log-uniform
    r = cell * 10 ** rng.uniform(-6, 0, n)
    s = t - d * r[:, None]
    s -= L * np.floor(s / L)
    ct, tl = _local(t, cell, nc)
    cs, sl = _local(s, cell, nc)
    o = cs - ct
    o -= nc * np.rint(o / nc).astype(np.int64)
    th, tlo = split(tl)
    sh, slo = split(sl)
    rh = ((th - o.astype(f32)).astype(f32) - sh).astype(f32)
    rl = (tlo - slo).astype(f32)
    r32 = ((rh + rl).astype(f32) * f32(cell)).astype(np.float64)
    exact = t - s
    exact -= L * np.rint(exact / L)
    err = np.linalg.norm(r32 - exact, axis=1) / np.linalg.norm(exact, axis=1)
    assert err.max() < 5e-7
