"""Proximal operator of tau TV + i_{>=0} by the fast gradient projection method (FGP).

Test infrastructure only.

Alg. 1 (Sec. 4.2) needs prox_{gamma tau R + i_{>=0}} with R the isotropic total variation; the paper
evaluates it with the fast gradient projection method of Beck and Teboulle (2009) on the dual problem.
Written from that method:

* discrete gradient D: forward differences along z, y, x with the difference set to 0 on the last
  plane of each axis (Neumann boundary); D^T = -div.
* dual variable p = (p_z, p_y, p_x) per voxel, feasible set |p(v)|_2 <= 1 (isotropic TV).
* for a dual point r:  x(r) = P_{>=0}(z + lam div r);  gradient step r + (1/(12 lam)) D x(r)
  (1/L with L = lam^2 ||D||^2 and ||D||^2 <= 12 in 3-D, scaled by lam as in Beck-Teboulle);
  projection of every voxel's 3-vector onto the unit ball; Nesterov extrapolation with
  t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2.
* the primal solution is x(p_K) after K iterations.
"""
from __future__ import annotations

import numpy as np


def grad3(x: np.ndarray) -> np.ndarray:
    """Forward differences (3, nz, ny, nx); zero on the last plane of each axis."""
    g = np.zeros((3,) + x.shape, dtype=np.float64)
    g[0, :-1] = x[1:] - x[:-1]
    g[1, :, :-1] = x[:, 1:] - x[:, :-1]
    g[2, :, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    return g


def div3(p: np.ndarray) -> np.ndarray:
    """Negative adjoint of grad3: <grad3 x, p> = -<x, div3 p>."""
    d = np.zeros(p.shape[1:], dtype=np.float64)
    d[:-1] += p[0, :-1]
    d[1:] -= p[0, :-1]
    d[:, :-1] += p[1, :, :-1]
    d[:, 1:] -= p[1, :, :-1]
    d[:, :, :-1] += p[2, :, :, :-1]
    d[:, :, 1:] -= p[2, :, :, :-1]
    return d


def tv(x: np.ndarray) -> float:
    """Isotropic total variation sum_v |D x (v)|_2."""
    return float(np.sqrt((grad3(x) ** 2).sum(axis=0)).sum())


def prox_tv_nonneg(z: np.ndarray, lam: float, iters: int) -> np.ndarray:
    """argmin_{x >= 0} 0.5 ||x - z||^2 + lam TV(x), approximated by `iters` FGP iterations."""
    z = np.asarray(z, dtype=np.float64)
    if lam <= 0:
        return np.maximum(z, 0.0)
    p = np.zeros((3,) + z.shape)
    r = p.copy()
    t = 1.0
    step = 1.0 / (12.0 * lam)
    for _ in range(iters):
        x = np.maximum(z + lam * div3(r), 0.0)
        q = r + step * grad3(x)
        q /= np.maximum(np.sqrt((q ** 2).sum(axis=0)), 1.0)
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        r = q + ((t - 1.0) / t_next) * (q - p)
        p, t = q, t_next
    return np.maximum(z + lam * div3(p), 0.0)
