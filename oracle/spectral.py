"""Plain numpy reference of the far-field pipeline of Sec. 2.2 (Algorithm 1,
steps P2G, FFT, CNV, IFFT, G2P) with the exact truncated Kaiser-Bessel window.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Loops follow the
definitions; numpy's FFT and Bessel I0 are used as library primitives.

Grid layout: ``grid[c, iz, iy, ix]`` is component c at the grid point
g = h * (ix, iy, iz), h = L / M (x fastest in memory).
"""
from __future__ import annotations

import numpy as np


def kb_params(P: int, h: float):
    """beta = 2.5 P and half-support a_w = P h / 2 (Sec. 2.2)."""
    return 2.5 * P, P * h / 2.0


def kb_window(t, P: int, h: float):
    """Truncated Kaiser-Bessel w_0(t) = I0(beta sqrt(1 - t^2/a_w^2)) / I0(beta)
    for |t| < a_w, else 0 (Sec. 2.2)."""
    beta, aw = kb_params(P, h)
    t = np.asarray(t, dtype=np.float64)
    inside = np.abs(t) < aw
    arg = np.sqrt(np.clip(1.0 - (t / aw) ** 2, 0.0, None))
    return np.where(inside, np.i0(beta * arg) / np.i0(beta), 0.0)


def kb_window_hat(k, P: int, h: float):
    """Fourier transform of the truncated KB window, int w_0(t) e^{-ikt} dt.

    The paper uses w-hat in eq. (sca) without printing it; this is the closed
    form of the transform of I0(beta sqrt(1 - x^2)) on [-1, 1]:
    2 a_w sinh(s)/(s I0(beta)), s = sqrt(beta^2 - (k a_w)^2), continued as
    2 a_w sin(s')/(s' I0(beta)), s' = sqrt((k a_w)^2 - beta^2), past k a_w = beta.
    """
    beta, aw = kb_params(P, h)
    k = np.asarray(k, dtype=np.float64)
    d = beta * beta - (k * aw) ** 2
    out = np.empty_like(k)
    pos, neg, zer = d > 0, d < 0, d == 0
    s = np.sqrt(d[pos])
    out[pos] = 2.0 * aw * np.sinh(s) / (s * np.i0(beta))
    s = np.sqrt(-d[neg])
    out[neg] = 2.0 * aw * np.sin(s) / (s * np.i0(beta))
    out[zer] = 2.0 * aw / np.i0(beta)
    return out


def _support_1d(y: float, P: int, h: float, M: int):
    """Grid indices l (unwrapped) with |l h - y| < a_w, their weights
    w_0(l h - y), and the wrapped indices l mod M."""
    _, aw = kb_params(P, h)
    lo = int(np.ceil((y - aw) / h))
    hi = int(np.floor((y + aw) / h))
    idx = np.arange(lo, hi + 1)
    w = kb_window(idx * h - y, P, h)
    return np.mod(idx, M), w


def spread(x, f, L: float, M: int, P: int) -> np.ndarray:
    """P2G, eq. (p2g): phi(g) = sum_j sum_p w(g - y_j + p) f_j."""
    h = L / M
    phi = np.zeros((3, M, M, M))
    for j in range(x.shape[0]):
        ix, wx = _support_1d(x[j, 0], P, h, M)
        iy, wy = _support_1d(x[j, 1], P, h, M)
        iz, wz = _support_1d(x[j, 2], P, h, M)
        w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
        Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
        for c in range(3):
            np.add.at(phi[c], (Z, Y, X), w * f[j, c])
    return phi


def gather(x, v, L: float, M: int, P: int) -> np.ndarray:
    """G2P, eq. (g2p): u(x_i) = h^3 sum_g sum_p w(x_i - g + p) v(g)."""
    h = L / M
    u = np.zeros((x.shape[0], 3))
    for i in range(x.shape[0]):
        ix, wx = _support_1d(x[i, 0], P, h, M)
        iy, wy = _support_1d(x[i, 1], P, h, M)
        iz, wz = _support_1d(x[i, 2], P, h, M)
        w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
        Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
        for c in range(3):
            u[i, c] = h ** 3 * np.sum(w * v[c][Z, Y, X])
    return u


def wave_numbers(L: float, M: int):
    """k = 2 pi m / L on the FFT grid, and a mask that drops k = 0 and, for
    even M, the Nyquist planes m = -M/2 (not representable symmetrically)."""
    m = np.fft.fftfreq(M, d=1.0 / M)  # integers in FFT order
    k1 = 2.0 * np.pi * m / L
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    MZ, MY, MX = np.meshgrid(m, m, m, indexing="ij")
    keep = ~((MX == 0) & (MY == 0) & (MZ == 0))
    if M % 2 == 0:
        nyq = -M // 2
        keep &= (MX != nyq) & (MY != nyq) & (MZ != nyq)
    return KX, KY, KZ, keep


def fourier_convolve(phi, L: float, M: int, P: int, xi: float) -> np.ndarray:
    """FFT -> CNV (eq. (sca): v-hat = Ghat^F / w-hat^2 * phi-hat) -> IFFT."""
    h = L / M
    ph = np.fft.fftn(phi, axes=(1, 2, 3))
    KX, KY, KZ, keep = wave_numbers(L, M)
    k = (KX, KY, KZ)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2s = np.where(keep, k2, 1.0)
    q = k2s / (2.0 * xi) ** 2
    # Ghat^F(k) of eq. (GFk), as 8 pi / k^4 (I k^2 - k k^T) e^{-q} (1 + q)
    s = 8.0 * np.pi / k2s ** 2 * np.exp(-q) * (1.0 + q)
    what2 = (kb_window_hat(KX, P, h) * kb_window_hat(KY, P, h) * kb_window_hat(KZ, P, h)) ** 2
    vh = np.zeros_like(ph)
    for a in range(3):
        acc = np.zeros_like(ph[0])
        for b in range(3):
            Gab = s * ((k2s if a == b else 0.0) - k[a] * k[b])
            acc = acc + Gab * ph[b]
        vh[a] = np.where(keep, acc / what2, 0.0)
    return np.real(np.fft.ifftn(vh, axes=(1, 2, 3)))


def far_field(x, f, L: float, M: int, P: int, xi: float) -> np.ndarray:
    """u^F_h at every point: the five steps of Sec. 2.2 in order."""
    phi = spread(x, f, L, M, P)
    v = fourier_convolve(phi, L, M, P, xi)
    return gather(x, v, L, M, P)
