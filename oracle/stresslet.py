"""CPU FP64 oracle for the double-layer (stresslet) part of the combined
single and double layer potential, Sec. 2.3.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Sec. 2.3 adds to eq. (potentials), for every source y_j with two vectors q_j
and n_j, the sum over sources and periodic images of T(x_i - y_j + p) applied
to q_j (x) n_j, where T is the stresslet (a symmetric 3x3x3 tensor) split as
T = T^N + T^F.  The paper leaves the form of T and of the split to another
work; the readings taken here are:

* T_jlm(r) = -6 r_j r_l r_m / |r|^5, the stresslet that goes with the
  Stokeslet G = I/|r| + r r^T/|r|^3 of Sec. 2 (the same normalisation), and
  u_j = sum_lm T_jlm D_lm with D = q (x) n (D_lm = q_l n_m).
* With phi = 1/|r|, T = 2 [d_m G_jl - delta_jl d_m phi + delta_jm d_l phi
  + delta_lm d_j phi].  The split screens every term the way eq. (g-near)
  screens G (Hasimoto: H(k) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)) on the
  Fourier side), which gives phi^N = erfc(xi r)/r - (xi/sqrt(pi)) e^{-xi^2 r^2}
  and, from G^N of eq. (g-near),
      T^N_jlm(r) = 2 beta(r) r_j r_l r_m
                   + 2 gamma(r) (delta_jl r_m + delta_jm r_l + delta_lm r_j),
      beta  = -3 erfc(xi r)/r^5 - (2 xi/sqrt(pi)) (3/r^4 + 2 xi^2/r^2) e^{-xi^2 r^2},
      gamma = (2 xi^3/sqrt(pi)) e^{-xi^2 r^2}.
  Any consistent split gives the same total; the tests pin this one by its
  xi-independence.
* Fourier side (f-hat(k) = int f(r) e^{-i k.r} dr):
      T-hat_jlm(k) = 8 pi i [(delta_jl k_m + delta_jm k_l + delta_lm k_j)/k^2
                             - 2 k_j k_l k_m / k^4],
  T-hat^F = H T-hat, and the k = 0 mode is dropped as for the Stokeslet.
  T^F is odd, so a target on a source needs no self term.
* Only the symmetric part of D enters (T is symmetric in l and m).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

from . import spectral

SQRT_PI = np.sqrt(np.pi)


def densities(q, n) -> np.ndarray:
    """D_j = q_j (x) n_j, shape (N, 3, 3) (D[j, l, m] = q[j, l] n[j, m])."""
    q = np.asarray(q, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return q[:, :, None] * n[:, None, :]


def apply_free(r, D) -> np.ndarray:
    """sum_lm T_jlm(r) D_lm for the bare stresslet, r (..., 3), D (..., 3, 3)."""
    r = np.asarray(r, dtype=np.float64)
    rr = np.sqrt(np.sum(r * r, axis=-1))
    rDr = np.einsum("...l,...lm,...m->...", r, D, r)
    return -6.0 * r * (rDr / rr ** 5)[..., None]


def near_coefficients(rr, xi: float):
    """beta(r), gamma(r) of T^N (module docstring)."""
    rr = np.asarray(rr, dtype=np.float64)
    e = np.exp(-(xi * rr) ** 2)
    beta = (-3.0 * erfc(xi * rr) / rr ** 5
            - (2.0 * xi / SQRT_PI) * (3.0 / rr ** 4 + 2.0 * xi ** 2 / rr ** 2) * e)
    gamma = (2.0 * xi ** 3 / SQRT_PI) * e
    return beta, gamma


def apply_near(r, D, xi: float) -> np.ndarray:
    """sum_lm T^N_jlm(r) D_lm = 2 beta r (r.D.r) + 2 gamma (r tr D + (D + D^T) r)."""
    r = np.asarray(r, dtype=np.float64)
    rr = np.sqrt(np.sum(r * r, axis=-1))
    beta, gamma = near_coefficients(rr, xi)
    rDr = np.einsum("...l,...lm,...m->...", r, D, r)
    tr = np.einsum("...ll->...", D)
    Ds = D + np.swapaxes(D, -1, -2)
    Dsr = np.einsum("...jm,...m->...j", Ds, r)
    return 2.0 * beta[..., None] * r * rDr[..., None] + 2.0 * gamma[..., None] * (r * tr[..., None] + Dsr)


def apply_fourier(k, Dh, xi: float | None) -> np.ndarray:
    """sum_lm T-hat_jlm(k) Dh_lm, times H(k) when xi is given (T-hat^F).
    k (..., 3) nonzero, Dh (..., 3, 3) complex; returns (..., 3) complex."""
    k = np.asarray(k, dtype=np.float64)
    k2 = np.sum(k * k, axis=-1)
    Ds = Dh + np.swapaxes(Dh, -1, -2)
    Dsk = np.einsum("...jm,...m->...j", Ds, k)
    tr = np.einsum("...ll->...", Dh)
    kDk = np.einsum("...l,...lm,...m->...", k, Dh, k)
    v = 8j * np.pi * ((Dsk + k * tr[..., None]) / k2[..., None] - 2.0 * k * (kDk / k2 ** 2)[..., None])
    if xi is not None:
        q = k2 / (4.0 * xi * xi)
        v = v * ((1.0 + q) * np.exp(-q))[..., None]
    return v


def default_xi(n: int, nt: int, L: float) -> float:
    """Balances real-space pairs against k-space modes; any xi gives the same sum."""
    xi = (3.0 * nt * n * np.pi ** 3 / max(n + nt, 1)) ** (1.0 / 6.0)
    return max(xi, 2.5) / L


def _images(reach: float, L: float):
    """Lattice shifts p with |p_c| <= reach + L/2 per component: every image
    within `reach` of a minimum-image difference (|d_c| <= L/2)."""
    m = int(np.floor(reach / L + 0.5 + 1e-9))
    g = np.arange(-m, m + 1)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return P * L


def near_field(x, D, L: float, xi: float, rc: float, targets=None) -> np.ndarray:
    """Real-space (P2P) sum of T^N over all sources and images with
    0 < |r| <= rc, at the targets (indices into x; all points if None).
    Differences are taken to the minimum image first, so only the shifts
    within rc + L/2 per component can reach."""
    x = np.asarray(x, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    tidx = np.arange(x.shape[0]) if targets is None else np.asarray(targets)
    shifts = _images(rc, L)
    u = np.zeros((len(tidx), 3))
    for a, i in enumerate(tidx):
        d = x[i] - x  # (n, 3)
        d -= L * np.round(d / L)
        for p in shifts:
            r = d + p
            rr2 = np.sum(r * r, axis=1)
            keep = (rr2 > 0.0) & (rr2 <= rc * rc)
            if np.any(keep):
                u[a] += apply_near(r[keep], D[keep], xi).sum(axis=0)
    return u


def wave_vectors(L: float, xi: float, kbox: int = 0):
    """k = 2 pi m / L, m != 0: inside the sphere |k| < 2 xi sqrt(40) (there
    H(k) < 1e-16), or with kbox > 0 the cube |m_d| <= kbox."""
    kcut = 2.0 * xi * np.sqrt(40.0)
    mmax = kbox if kbox > 0 else int(np.ceil(kcut * L / (2.0 * np.pi)))
    g = np.arange(-mmax, mmax + 1)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    k = 2.0 * np.pi * m / L
    k2 = np.sum(k * k, axis=1)
    keep = k2 > 0.0
    if kbox <= 0:
        keep &= k2 < kcut * kcut
    return k[keep]


def far_field(x, D, L: float, xi: float, targets=None, kbox: int = 0,
              chunk: int = 4096) -> np.ndarray:
    """(1/V) sum_{k != 0} T-hat^F(k) : D-hat(k) e^{i k.x} at the targets, with
    D-hat(k) = sum_j D_j e^{-i k.y_j} (direct k sum, no grid)."""
    x = np.asarray(x, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    tidx = np.arange(x.shape[0]) if targets is None else np.asarray(targets)
    kv = wave_vectors(L, xi, kbox)
    u = np.zeros((len(tidx), 3))
    for s in range(0, len(kv), chunk):
        k = kv[s:s + chunk]
        ph = np.exp(-1j * (x @ k.T))                     # (n, nk)
        Dh = np.einsum("jk,jlm->klm", ph, D)             # (nk, 3, 3)
        v = apply_fourier(k, Dh, xi)                     # (nk, 3)
        et = np.exp(1j * (x[tidx] @ k.T))                # (nt, nk)
        u += np.real(et @ v)
    return u / L ** 3


def ewald(x, D, L: float, xi: float | None = None, targets=None) -> np.ndarray:
    """The double-layer periodic sum at the targets: T^N over all images
    within exp(-xi^2 r^2) < 1e-18 plus the direct k sum of T^F."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    nt = n if targets is None else len(targets)
    if xi is None:
        xi = default_xi(n, nt, L)
    rmax = 6.5 / xi
    return near_field(x, D, L, xi, rmax, targets) + far_field(x, D, L, xi, targets)


def symmetric_parts(D) -> tuple[np.ndarray, np.ndarray]:
    """The six independent components of (D + D^T)/2 as two triples:
    (D_xx, D_yy, D_zz) and (D_xy, D_xz, D_yz)."""
    S = 0.5 * (D + np.swapaxes(D, -1, -2))
    return (np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2]], axis=1),
            np.stack([S[:, 0, 1], S[:, 0, 2], S[:, 1, 2]], axis=1))


def far_field_spectral(x, D, L: float, M: int, P: int, xi: float) -> np.ndarray:
    """The grid form of far_field, the steps of Sec. 2.2 with the double
    layer's six symmetric density components (Sec. 2.3): spread (P2G), FFT,
    CNV with T-hat^F / w-hat^2, IFFT, gather (G2P)."""
    x = np.asarray(x, dtype=np.float64)
    dd, od = symmetric_parts(np.asarray(D, dtype=np.float64))
    phd = np.fft.fftn(spectral.spread(x, dd, L, M, P), axes=(1, 2, 3))
    pho = np.fft.fftn(spectral.spread(x, od, L, M, P), axes=(1, 2, 3))
    h = L / M
    KX, KY, KZ, keep = spectral.wave_numbers(L, M)
    k = np.stack([KX, KY, KZ], axis=-1)
    k[~keep] = 1.0  # placeholder, zeroed below
    Dh = np.empty(KX.shape + (3, 3), dtype=np.complex128)
    Dh[..., 0, 0], Dh[..., 1, 1], Dh[..., 2, 2] = phd[0], phd[1], phd[2]
    Dh[..., 0, 1] = Dh[..., 1, 0] = pho[0]
    Dh[..., 0, 2] = Dh[..., 2, 0] = pho[1]
    Dh[..., 1, 2] = Dh[..., 2, 1] = pho[2]
    v = apply_fourier(k, Dh, xi)
    what2 = (spectral.kb_window_hat(KX, P, h) * spectral.kb_window_hat(KY, P, h)
             * spectral.kb_window_hat(KZ, P, h)) ** 2
    v = np.where(keep[..., None], v / what2[..., None], 0.0)
    vg = np.real(np.fft.ifftn(np.moveaxis(v, -1, 0), axes=(1, 2, 3)))
    return spectral.gather(x, vg, L, M, P)


def coulomb_potential(xe, y, c, L: float, xi: float) -> np.ndarray:
    """Periodic Coulomb potential sum_j sum_p c_j / |xe - y_j + p| at points xe
    that are not sources, by the textbook Ewald split (erfc(xi r)/r in real
    space, 4 pi/(V k^2) e^{-k^2/(4 xi^2)} in k space, k = 0 dropped).  An
    independent routine: the double layer with D = I at every source is
    6 grad of this potential (T_jll = -6 r_j/r^3 = 6 d_j (1/r))."""
    xe = np.atleast_2d(np.asarray(xe, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    rmax = 6.5 / xi
    shifts = _images(rmax, L)
    phi = np.zeros(xe.shape[0])
    for a, xa in enumerate(xe):
        d = xa - y
        d -= L * np.round(d / L)  # minimum image; shifts reach rmax + L/2
        for p in shifts:
            rr = np.sqrt(np.sum((d + p) ** 2, axis=1))
            m = (rr > 0.0) & (rr < rmax)
            phi[a] += np.sum(c[m] * erfc(xi * rr[m]) / rr[m])
    kv = wave_vectors(L, xi)
    k2 = np.sum(kv * kv, axis=1)
    S = c @ np.exp(-1j * (y @ kv.T))  # (nk,)
    g = 4.0 * np.pi / k2 * np.exp(-k2 / (4.0 * xi * xi)) * S
    phi += np.real(np.exp(1j * (xe @ kv.T)) @ g) / L ** 3
    return phi


def coulomb_site_potential(y, c, L: float, xi: float) -> np.ndarray:
    """Potential at each charge from all the others (and their images), the
    point's own image charges included: the Ewald sum with the self term
    -2 xi c_i / sqrt(pi) removed.  The charges must sum to zero."""
    y = np.asarray(y, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    rmax = 6.5 / xi
    shifts = _images(rmax, L)
    phi = np.zeros(y.shape[0])
    for i in range(y.shape[0]):
        d = y[i] - y
        d -= L * np.round(d / L)  # minimum image; shifts reach rmax + L/2
        for p in shifts:
            rr = np.sqrt(np.sum((d + p) ** 2, axis=1))
            m = (rr > 0.0) & (rr < rmax)
            phi[i] += np.sum(c[m] * erfc(xi * rr[m]) / rr[m])
    kv = wave_vectors(L, xi)
    k2 = np.sum(kv * kv, axis=1)
    S = c @ np.exp(-1j * (y @ kv.T))
    g = 4.0 * np.pi / k2 * np.exp(-k2 / (4.0 * xi * xi)) * S
    phi += np.real(np.exp(1j * (y @ kv.T)) @ g) / L ** 3
    return phi - 2.0 * xi * c / SQRT_PI
