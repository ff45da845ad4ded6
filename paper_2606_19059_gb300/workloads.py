"""Seeded synthetic inputs: point clouds in a cubic box and force densities.

This module holds no Ewald arithmetic; the tests, the oracle checks and the
benchmark all draw their inputs from it, so both sides of every parity check
see identical points and forces.  Distributions follow the paper's synthetic
workloads (Sec. 6 and App. B: uniform, truncated normal, clustered), with the
clustered case made periodic (blobs wrap around the box).
"""
from __future__ import annotations

import numpy as np


def forces(rng: np.random.Generator, n: int, zero_mean: bool = True) -> np.ndarray:
    """Force densities f ~ N(0, 1) per component, optionally minus their mean."""
    f = rng.standard_normal((n, 3))
    if zero_mean and n > 1:
        f -= f.mean(axis=0, keepdims=True)
    return f


def uniform(rng: np.random.Generator, n: int, L: float = 1.0) -> np.ndarray:
    """n points uniform in [0, L)^3."""
    return rng.random((n, 3)) * L


def clustered(rng: np.random.Generator, n: int, L: float = 1.0, n_blobs: int = 200,
              sigma: float = 0.02, background: float = 0.2) -> np.ndarray:
    """Gaussian blobs (std sigma*L, centres uniform, wrapped periodically) plus
    a uniform background fraction; returned in shuffled order."""
    n_bg = int(round(background * n))
    n_bl = n - n_bg
    centres = rng.random((n_blobs, 3)) * L
    owner = np.arange(n_bl) % n_blobs
    pts = centres[owner] + rng.standard_normal((n_bl, 3)) * (sigma * L)
    pts = np.concatenate([pts, rng.random((n_bg, 3)) * L])
    pts = np.mod(pts, L)
    pts[pts >= L] = 0.0  # guard the mod rounding to exactly L
    return pts[rng.permutation(n)]


def make(kind: str, n: int, seed: int, L: float = 1.0):
    """(x, f) for a named distribution: 'uniform' or 'clustered'."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        x = uniform(rng, n, L)
    elif kind == "clustered":
        x = clustered(rng, n, L)
    else:
        raise ValueError(f"unknown distribution {kind!r}")
    return x, forces(rng, n)


# Named workloads: (distribution, N, L, tol, grid M or None, support P or None, seed)
WORKLOADS = {
    "uniform_1e3_tol1e-8": ("uniform", 1000, 1.0, 1e-8, None, None, 1001),
    "uniform_1e5_tol1e-6_M128_P12": ("uniform", 100_000, 1.0, 1e-6, 128, 12, 1002),
    "clustered_2e6_tol1e-7_M256_P14": ("clustered", 2_000_000, 1.0, 1e-7, 256, 14, 1003),
}


# Many independent boxes: N = round(10^U(log10 n_lo, log10 n_hi)) per box,
# tol drawn uniformly from `tols`, uniform points in the unit box and
# zero-mean forces.  Box b's own points come from seed (seed, b).
BATCH_TOLS = (1e-4, 1e-6, 1e-8)


def batch_boxes(nbox: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e5, tols=BATCH_TOLS):
    """Sizes and tolerances of `nbox` boxes: (N array int64, tol array)."""
    rng = np.random.default_rng(seed)
    N = np.rint(10.0 ** rng.uniform(np.log10(n_lo), np.log10(n_hi), nbox)).astype(np.int64)
    tol = np.asarray(tols, dtype=np.float64)[rng.integers(0, len(tols), nbox)]
    return N, tol


def batch_box(seed: int, b: int, n: int, L: float = 1.0):
    """(x, f) of box b of a batch drawn with `seed`: uniform points, forces."""
    rng = np.random.default_rng([seed, b])
    return uniform(rng, n, L), forces(rng, n)


# Served requests: f_t = f_{t-1} + a n_t re-centred, n_t ~ N(0, 1) from the
# counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011),
# written from its published definition: counter (i mod 2^32, i div 2^32, t, 0)
# for point i, key (seed mod 2^32, seed div 2^32), ten rounds; outputs
# (c0, c1) -> u1, u2 = (c + 1) / 2^32 and Box-Muller n_x, n_y =
# sqrt(-2 ln u1) (cos, sin)(2 pi u2); (c2, c3) likewise give n_z (cosine).
_PHILOX_M = (0xD2511F53, 0xCD9E8D57)
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Ten Philox4x32 rounds on uint32 counters (arrays) under key (k0, k1)."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3)]
    k0, k1 = np.uint64(k0 & 0xFFFFFFFF), np.uint64(k1 & 0xFFFFFFFF)
    m0, m1 = np.uint64(_PHILOX_M[0]), np.uint64(_PHILOX_M[1])
    for _ in range(10):
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(_PHILOX_W[0])) & _MASK32
        k1 = (k1 + np.uint64(_PHILOX_W[1])) & _MASK32
    return c


def perturbation_normals(n: int, step: int, seed: int) -> np.ndarray:
    """The (n, 3) standard normals of update `step` of a request with `seed`."""
    i = np.arange(n, dtype=np.uint64)
    c = philox4x32_10(i & _MASK32, i >> np.uint64(32), np.full(n, step, dtype=np.uint64),
                      np.zeros(n, dtype=np.uint64), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = [(v.astype(np.float64) + 1.0) / 4294967296.0 for v in c]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    t0, t1 = 2.0 * np.pi * u[1], 2.0 * np.pi * u[3]
    return np.stack([r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1)], axis=1)


def served_forces(f0: np.ndarray, napplies: int, perturb: float, seed: int) -> np.ndarray:
    """The forces of the last of `napplies` applies of a served request."""
    f = np.array(f0, dtype=np.float64, copy=True)
    for t in range(1, napplies):
        f = f + perturb * perturbation_normals(f.shape[0], t, seed)
        f -= f.mean(axis=0, keepdims=True)
    return f


def serving_stream(nreq: int, seed: int, rate_hz: float, n_lo: float = 1e3, n_hi: float = 4e6,
                   tols=BATCH_TOLS):
    """Poisson arrivals: list of dicts (t arrival in s, N, kind, tol, seed)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, nreq))
    N = np.rint(10.0 ** rng.uniform(np.log10(n_lo), np.log10(n_hi), nreq)).astype(np.int64)
    kinds = np.where(rng.random(nreq) < 0.5, "uniform", "clustered")
    tol = np.asarray(tols, dtype=np.float64)[rng.integers(0, len(tols), nreq)]
    return [{"t": float(t[i]), "N": int(N[i]), "kind": str(kinds[i]), "tol": float(tol[i]),
             "seed": int(seed * 100003 + i)} for i in range(nreq)]


def served_box(kind: str, n: int, seed: int, L: float = 1.0):
    """(x, f0) of a served request: uniform, or clustered with blobs in
    proportion to N (one per 10^4 points, at least one), same sigma and 20%
    background."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        x = uniform(rng, n, L)
    else:
        x = clustered(rng, n, L, n_blobs=max(1, int(round(n / 1e4))))
    return x, forces(rng, n)
