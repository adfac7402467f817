"""Scalar scattering of a plane wave by a homogeneous sphere (partial waves; oracle).

The paper validates its forward model against the analytic field of a bead
(Sec. 3.1, Fig. 3).  For the scalar Helmholtz equation that field is the
partial-wave series below.  With f = k_b^2((eta/eta_b)^2 - 1) the LS equation
(eq. lipp) is equivalent to  Laplace(u) + k^2 u = 0  with k = k_1 = k_b eta/eta_b
inside the sphere and k_b outside, plus the outgoing radiation condition.

Incident wave exp(i k_b z) = sum_l i^l (2l+1) j_l(k_b r) P_l(cos theta).
Outside:  u = exp(i k_b z) + sum_l i^l (2l+1) a_l h_l(k_b r) P_l(cos theta)
Inside:   u = sum_l i^l (2l+1) c_l j_l(k_1 r) P_l(cos theta)
a_l, c_l from continuity of u and du/dr at r = a.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def coefficients(radius: float, kb: float, k1: float, lmax: int | None = None):
    x, y = kb * radius, k1 * radius
    if lmax is None:
        lmax = int(np.ceil(max(x, y) + 4.0 * max(x, y) ** (1.0 / 3.0) + 10))
    l = np.arange(lmax + 1)
    jx, djx = spherical_jn(l, x), spherical_jn(l, x, derivative=True)
    yx, dyx = spherical_yn(l, x), spherical_yn(l, x, derivative=True)
    jy, djy = spherical_jn(l, y), spherical_jn(l, y, derivative=True)
    hx, dhx = jx + 1j * yx, djx + 1j * dyx
    a = (k1 * djy * jx - kb * djx * jy) / (kb * jy * dhx - k1 * djy * hx)
    c = (jx + a * hx) / jy
    return l, a, c


def total_field(px, py, pz, radius: float, kb: float, k1: float, lmax: int | None = None):
    """Total field at points (px, py, pz) (arrays, micrometres) for a sphere centred at the origin."""
    px, py, pz = np.broadcast_arrays(np.asarray(px, float), np.asarray(py, float), np.asarray(pz, float))
    r = np.sqrt(px * px + py * py + pz * pz)
    cos_t = np.where(r > 0, pz / np.where(r > 0, r, 1.0), 1.0)
    l, a, c = coefficients(radius, kb, k1, lmax)
    inside = r < radius
    out = np.where(inside, 0.0 + 0j, np.exp(1j * kb * pz))
    for li, al, cl in zip(l, a, c):
        P = eval_legendre(li, cos_t)
        pref = (1j ** li) * (2 * li + 1)
        hin = spherical_jn(li, k1 * r)
        hout = spherical_jn(li, kb * r) + 1j * spherical_yn(li, np.where(r > 0, kb * r, 1.0))
        out = out + np.where(inside, pref * cl * hin * P, pref * al * hout * P)
    return out
