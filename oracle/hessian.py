"""Proximal operator of tau ||H .||_{S1,1} + i_{>=0}: the Hessian Schatten-norm regulariser of Alg. 1.

Test infrastructure only.

Sec. 4.2 names the Hessian Schatten-norm regulariser (Lefkimmiatis et al. 2013) as the alternative
to TV and evaluates its prox with the extension of FGP to it.  Written from that method:

* discrete Hessian H x (v) = [D_ab x (v)]_{a,b in (z, y, x)}, symmetric 3 x 3 per voxel, with
  D_aa = -D_a^T D_a (second difference, Neumann boundary) and D_ab = D_b D_a for a != b, D_a the
  forward difference of the TV prox (zero on the last plane of axis a).  Fields of symmetric
  matrices are stored as 6 components (zz, yy, xx, zy, zx, yx) with the Frobenius inner product
  (off-diagonal components counted twice), so H^* = sum_a D_aa Psi_aa + 2 sum_{a<b} D_a^T D_b^T Psi_ab.
* ||H||^2 <= 3 * 16 + 6 * 16 = 144 (||D_aa|| <= 4, ||D_ab|| <= 4).
* the regulariser is the sum over voxels of the nuclear norm (Schatten 1-norm) of H x (v); its dual
  ball is the spectral-norm (Schatten infinity) unit ball, onto which a symmetric matrix is
  projected by clipping its eigenvalues to [-1, 1].
* FGP on the dual: x(W) = P_{>=0}(z - lam H^* W); Psi = P_ball(W + (1/(144 lam)) H x(W));
  Nesterov extrapolation as in the TV prox; the result is x(Psi_K).
"""
from __future__ import annotations

import numpy as np

from .tv import grad3

# component order and Frobenius weights
COMPONENTS = ("zz", "yy", "xx", "zy", "zx", "yx")
WEIGHTS = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


def _d(x: np.ndarray, axis: int) -> np.ndarray:
    """Forward difference along `axis`, zero on the last plane."""
    return grad3(x)[axis] if x.ndim == 3 else None


def _dt(p: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint of the forward difference: (D^T p)[i] = p[i-1] [i >= 1] - p[i] [i <= n-2]."""
    out = np.zeros_like(p)
    n = p.shape[axis]
    sl = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(3))  # noqa: E731
    out[sl(1, n)] += p[sl(0, n - 1)]
    out[sl(0, n - 1)] -= p[sl(0, n - 1)]
    return out


def hessian(x: np.ndarray) -> np.ndarray:
    """H x as (6, nz, ny, nx) in the order zz, yy, xx, zy, zx, yx."""
    x = np.asarray(x, dtype=np.float64)
    d = [_d(x, a) for a in range(3)]
    out = np.empty((6,) + x.shape)
    for a in range(3):
        out[a] = -_dt(d[a], a)
    out[3] = _d(d[0], 1)   # D_y D_z
    out[4] = _d(d[0], 2)   # D_x D_z
    out[5] = _d(d[1], 2)   # D_x D_y
    return out


def hessian_adjoint(w: np.ndarray) -> np.ndarray:
    """H^* with respect to the weighted (Frobenius) inner product of symmetric-matrix fields."""
    out = np.zeros(w.shape[1:])
    for a in range(3):
        out -= _dt(_d(w[a], a), a)     # D_aa is symmetric
    out += 2.0 * _dt(_dt(w[3], 1), 0)
    out += 2.0 * _dt(_dt(w[4], 2), 0)
    out += 2.0 * _dt(_dt(w[5], 2), 1)
    return out


def field_dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.tensordot(WEIGHTS, (a * b).reshape(6, -1).sum(axis=1), axes=1))


def to_matrices(w: np.ndarray) -> np.ndarray:
    """(6, ...) -> (..., 3, 3) symmetric matrices."""
    zz, yy, xx, zy, zx, yx = w
    m = np.empty(w.shape[1:] + (3, 3))
    m[..., 0, 0], m[..., 1, 1], m[..., 2, 2] = zz, yy, xx
    m[..., 0, 1] = m[..., 1, 0] = zy
    m[..., 0, 2] = m[..., 2, 0] = zx
    m[..., 1, 2] = m[..., 2, 1] = yx
    return m


def from_matrices(m: np.ndarray) -> np.ndarray:
    return np.stack([m[..., 0, 0], m[..., 1, 1], m[..., 2, 2], m[..., 0, 1], m[..., 0, 2], m[..., 1, 2]])


def project_spectral_ball(w: np.ndarray) -> np.ndarray:
    """Every voxel's symmetric matrix onto {||M||_2 <= 1}: eigenvalues clipped to [-1, 1]."""
    m = to_matrices(w)
    vals, vecs = np.linalg.eigh(m)
    vals = np.clip(vals, -1.0, 1.0)
    return from_matrices(np.einsum("...ij,...j,...kj->...ik", vecs, vals, vecs))


def hs1(x: np.ndarray) -> float:
    """sum_v ||H x (v)||_{S1} (nuclear norm of every voxel's Hessian)."""
    return float(np.abs(np.linalg.eigvalsh(to_matrices(hessian(x)))).sum())


def prox_hs_nonneg(z: np.ndarray, lam: float, iters: int) -> np.ndarray:
    """argmin_{x >= 0} 0.5 ||x - z||^2 + lam sum_v ||H x (v)||_{S1}, by `iters` FGP iterations."""
    z = np.asarray(z, dtype=np.float64)
    if lam <= 0:
        return np.maximum(z, 0.0)
    p = np.zeros((6,) + z.shape)
    r = p.copy()
    t = 1.0
    step = 1.0 / (144.0 * lam)
    for _ in range(iters):
        x = np.maximum(z - lam * hessian_adjoint(r), 0.0)
        q = project_spectral_ball(r + step * hessian(x))
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        r = q + ((t - 1.0) / t_next) * (q - p)
        p, t = q, t_next
    return np.maximum(z - lam * hessian_adjoint(p), 0.0)
