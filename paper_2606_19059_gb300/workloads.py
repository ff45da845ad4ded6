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
