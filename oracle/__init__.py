"""CPU FP64 oracle for the triply periodic Stokeslet Ewald sum.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The CUDA library
never loads it, and it shares no code with the library.

Contents
--------
* ``ewald_oracle.c`` (plain C, FP64, OpenMP): the direct Ewald sum, the
  near-field (P2P) reference, the direct k-space far field and a brute-force
  image sum of the bare Stokeslet.  Built here with gcc into ``_oracle.so``.
* ``spectral.py`` (numpy): the far-field pipeline of Sec. 2.2 (P2G, FFT,
  CNV, IFFT, G2P) with the exact truncated Kaiser-Bessel window.
* ``stresslet.py`` (numpy): the double-layer (stresslet) part of the combined
  potential of Sec. 2.3 -- direct Ewald sum, near-field reference and the
  grid pipeline -- and a textbook Coulomb Ewald sum that pins it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald_oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ewald_oracle.c with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_ewald.argtypes = [i64, d, p, p, d, i64, p, p]
        lib.oracle_near_field.argtypes = [i64, d, p, p, d, d, p]
        lib.oracle_far_field.argtypes = [i64, d, p, p, d, i64, i64, p, p]
        lib.oracle_image_sum.argtypes = [i64, d, p, p, d, p]
        for fn in (lib.oracle_ewald, lib.oracle_near_field, lib.oracle_far_field,
                   lib.oracle_image_sum, lib.oracle_num_threads):
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def default_xi(n: int, nt: int, L: float) -> float:
    """A splitting parameter that balances the oracle's real-space work
    (nt * n * sphere volume) against its k-space work (modes * (n + nt)).
    Any xi gives the same converged sum; this only sets the running time."""
    xi = (3.0 * nt * n * np.pi ** 3 / max(n + nt, 1)) ** (1.0 / 6.0)
    return max(xi, 2.5) / L


def ewald(x, f, L: float, xi: float | None = None, targets=None) -> np.ndarray:
    """Direct Ewald sum u at the target indices (all points if None), FP64."""
    x, f = _c(x), _c(f)
    n = x.shape[0]
    tidx = None if targets is None else _c(targets, np.int64)
    nt = n if tidx is None else tidx.shape[0]
    if xi is None:
        xi = default_xi(n, nt, L)
    u = np.zeros((nt, 3))
    rc = _load().oracle_ewald(n, L, x.ctypes.data, f.ctypes.data, float(xi), nt,
                              None if tidx is None else tidx.ctypes.data, u.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_ewald failed")
    return u


def near_field(x, f, L: float, xi: float, rc: float) -> np.ndarray:
    """Near-field (P2P) sum with cutoff |r| <= rc at every point."""
    x, f = _c(x), _c(f)
    u = np.zeros_like(x)
    _load().oracle_near_field(x.shape[0], L, x.ctypes.data, f.ctypes.data, float(xi),
                              float(rc), u.ctypes.data)
    return u


def far_field(x, f, L: float, xi: float, kbox: int = 0, targets=None) -> np.ndarray:
    """Far field by direct k sum (no self term removed)."""
    x, f = _c(x), _c(f)
    n = x.shape[0]
    tidx = None if targets is None else _c(targets, np.int64)
    nt = n if tidx is None else tidx.shape[0]
    u = np.zeros((nt, 3))
    rc = _load().oracle_far_field(n, L, x.ctypes.data, f.ctypes.data, float(xi), int(kbox), nt,
                                  None if tidx is None else tidx.ctypes.data, u.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_far_field failed")
    return u


def image_sum(x, f, L: float, R: float) -> np.ndarray:
    """Brute-force spherical image sum of the bare Stokeslet, radius R."""
    x, f = _c(x), _c(f)
    u = np.zeros_like(x)
    _load().oracle_image_sum(x.shape[0], L, x.ctypes.data, f.ctypes.data, float(R),
                             u.ctypes.data)
    return u


def self_coefficient(xi: float) -> float:
    """lim_{r->0} (G - G^N) = (4 xi / sqrt(pi)) I, from eq. (g-near)."""
    return 4.0 * xi / np.sqrt(np.pi)
