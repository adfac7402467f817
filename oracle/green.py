"""Green function pieces of the LS model (oracle; test infrastructure only).

Sec. 2.1: scattering potential and free-space Green function.
Sec. 3.1: truncated Green function g_t and its Fourier transform (eq. GreenL,
eq. GreenL2).
"""
from __future__ import annotations

import numpy as np


def wavenumber(lam_um: float, eta_b: float) -> float:
    """k_b = 2 pi eta_b / lambda (Sec. 2.1)."""
    return 2.0 * np.pi * eta_b / lam_um


def scattering_potential(dn: np.ndarray, eta_b: float, lam_um: float) -> np.ndarray:
    """f = k_b^2 ((eta / eta_b)^2 - 1) with eta = eta_b + dn (Sec. 2.1)."""
    kb = wavenumber(lam_um, eta_b)
    eta = eta_b + np.asarray(dn, dtype=np.float64)
    return kb * kb * ((eta / eta_b) ** 2 - 1.0)


def green(r: np.ndarray, kb: float) -> np.ndarray:
    """Outgoing free-space Green function g(x) = exp(i k_b |x|) / (4 pi |x|) (eq. def:Green)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(1j * kb * r) / (4.0 * np.pi * r)


def truncation_radius(lengths) -> float:
    """Radius of the support of g_t: the diagonal of Omega (sqrt(3) L for a cube, Sec. 3.1)."""
    return float(np.sqrt(np.sum(np.asarray(lengths, dtype=np.float64) ** 2)))


def _sinc(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0.0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def ghat_t(w, kb: float, R: float, *, _sinc_sign: float = -1.0):
    """Fourier transform of the truncated Green function at radial frequency ``w`` = ||omega||.

    eq. GreenL (for ||w|| != k_b):
        ghat_t(w) = [1 - e^{i k_b R} (cos(R w) - i k_b R sinc(R w))] / (w^2 - k_b^2)
    eq. GreenL2 (continuous extension at ||w|| = k_b):
        ghat_t(k_b) = i (R / (2 k_b) - e^{i k_b R} sin(k_b R) / (2 k_b^2))
    with R the truncation radius (sqrt(3) L in the paper).

    ``_sinc_sign`` is the sign in front of the sinc term.  -1 is the reading
    used everywhere (see the package docstring); +1 reproduces the sign as
    printed and exists only so that a test can show that the quadrature pin
    rejects it.

    Within |w - k_b| < 1e-8 / R the formula loses accuracy to cancellation
    (0/0); there the GreenL2 value is used (its truncation error at that
    distance is below 1e-8 relative).
    """
    w = np.asarray(w, dtype=np.float64)
    e = np.exp(1j * kb * R)
    num = 1.0 - e * (np.cos(R * w) + _sinc_sign * 1j * kb * R * _sinc(R * w))
    den = w * w - kb * kb
    near = np.abs(w - kb) < 1e-8 / R
    safe_den = np.where(near, 1.0, den)
    val = num / safe_den
    at_kb = 1j * (R / (2.0 * kb) - e * np.sin(kb * R) / (2.0 * kb * kb))
    return np.where(near, at_kb, val)


def ghat_t_zero(kb: float, R: float) -> complex:
    """Closed form of ghat_t(0) = integral of g over the ball of radius R:
    (e^{i k_b R}(1 - i k_b R) - 1) / k_b^2 (derived from the definition of g_t)."""
    e = np.exp(1j * kb * R)
    return (e * (1.0 - 1j * kb * R) - 1.0) / (kb * kb)


def ghat_t_quadrature(w, kb: float, R: float, nodes: int = 4000) -> np.ndarray:
    """Independent numeric evaluation of the Fourier transform of g_t (no closed form used).

    For a radial function supported on the ball of radius R,
        ghat_t(w) = 4 pi int_0^R g(r) r^2 sinc(w r) dr = int_0^R e^{i k_b r} r sinc(w r) dr,
    evaluated by Gauss-Legendre quadrature on [0, R] split into panels.
    """
    w = np.atleast_1d(np.asarray(w, dtype=np.float64))
    x, wt = np.polynomial.legendre.leggauss(64)
    panels = max(1, nodes // 64)
    edges = np.linspace(0.0, R, panels + 1)
    r = ((edges[1:, None] - edges[:-1, None]) * 0.5 * x[None, :] + 0.5 * (edges[1:, None] + edges[:-1, None])).ravel()
    dr = (((edges[1:] - edges[:-1]) * 0.5)[:, None] * wt[None, :]).ravel()
    f = np.exp(1j * kb * r) * r
    out = np.empty(w.shape, dtype=np.complex128)
    for i, wi in enumerate(w):
        out[i] = np.sum(f * _sinc(wi * r) * dr)
    return out
