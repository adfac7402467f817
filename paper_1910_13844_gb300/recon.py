"""Variational reconstruction on top of the LS model (Sec. 4, Alg. 1).

    f* in argmin_f  sum_q ||H_q(f) - y_q||^2 / (2 ||y_q||^2) + tau TV(f) + i_{>=0}(f)   (eq. prob)

solved by accelerated forward-backward splitting (FISTA, Alg. 1) with step
gamma_k = gamma_0 / sqrt(k), optional random view subsets per iteration
(Alg. 1 line 5), and the proximal operator of gamma tau TV + i_{>=0} evaluated
by the fast gradient projection method (FGP) on the dual of isotropic TV.
The data-term gradient (Alg. 1 line 6) comes from the CUDA library, batched
over the selected views (or one view per call, for comparison); the TV prox
and the FISTA updates are element-wise tensor operations on the device.

Reading of Alg. 1: the gradient is evaluated at the extrapolated point v^k
(standard FISTA), where the listing writes f^k.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ls_forward, ls_gradient, ls_plane_waves, ls_residual


# ------------------------------------------------------------------ TV prox (FGP)
def _grad3(x):
    """Forward differences with Neumann boundary, stacked (3, nz, ny, nx)."""
    g = torch.zeros((3,) + x.shape, dtype=x.dtype, device=x.device)
    g[0, :-1] = x[1:] - x[:-1]
    g[1, :, :-1] = x[:, 1:] - x[:, :-1]
    g[2, :, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    return g


def _div3(p):
    """Negative adjoint of _grad3."""
    d = torch.zeros(p.shape[1:], dtype=p.dtype, device=p.device)
    d[:-1] += p[0, :-1]
    d[1:] -= p[0, :-1]
    d[:, :-1] += p[1, :, :-1]
    d[:, 1:] -= p[1, :, :-1]
    d[:, :, :-1] += p[2, :, :, :-1]
    d[:, :, 1:] -= p[2, :, :, :-1]
    return d


def prox_tv_nonneg(z: torch.Tensor, lam: float, iters: int = 20) -> torch.Tensor:
    """argmin_x 0.5 ||x - z||^2 + lam TV(x) + i_{>=0}(x) by FGP (Beck and Teboulle 2009)."""
    if lam <= 0:
        return z.clamp_min(0.0)
    p = torch.zeros((3,) + z.shape, dtype=z.dtype, device=z.device)
    r = p.clone()
    t = 1.0
    step = 1.0 / (12.0 * lam)          # 1 / (lam * ||grad||^2), ||grad||^2 <= 12 in 3-D
    for _ in range(iters):
        x = (z + lam * _div3(r)).clamp_min(0.0)
        pn = r + step * _grad3(x)
        norm = pn.pow(2).sum(dim=0).sqrt().clamp_min(1.0)
        pn = pn / norm
        tn = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        r = pn + ((t - 1.0) / tn) * (pn - p)
        p, t = pn, tn
    return (z + lam * _div3(p)).clamp_min(0.0)


# ------------------------------------------------------------------ data term
@dataclass
class Problem:
    plan: object                 # paper_1910_13844_gb300.Plan
    kvec: np.ndarray             # (Q, 3) wave vectors
    y: torch.Tensor              # (Q, my, mx) measurements
    weights: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.weights is None:
            yy = self.y.reshape(self.y.shape[0], -1).abs().pow(2).sum(dim=1).double().cpu().numpy()
            self.weights = 1.0 / yy


def data_grad(prob: Problem, f: torch.Tensor, views=None, batched: bool = True):
    """(loss, gradient) of the data term over `views` (all if None): batched, or one view per call."""
    Q = prob.kvec.shape[0]
    idx = list(range(Q)) if views is None else list(views)
    plan = prob.plan
    groups = [idx] if batched else [[q] for q in idx]
    grad = torch.zeros_like(f)
    loss = 0.0
    for g in groups:
        k = prob.kvec[g]
        uin = plan.field(len(g))
        ls_plane_waves(plan.handle, k, uin)
        u = plan.field(len(g))
        far = plan.detector(len(g))
        ls_forward(plan.handle, f, uin, u, far)
        res = torch.empty_like(far)
        y = prob.y[g].contiguous()
        l2 = ls_residual(far, y, res)
        w = prob.weights[g]
        loss += 0.5 * float(np.sum(l2 * w))
        gq = torch.empty_like(f)
        ls_gradient(plan.handle, f, res, gq, u_fwd=u, view_weights=w)
        grad += gq
    return loss, grad


# ------------------------------------------------------------------ FISTA (Alg. 1)
@dataclass
class FistaState:
    f: torch.Tensor
    f_prev: torch.Tensor
    v: torch.Tensor
    alpha: float = 1.0
    k: int = 1
    history: list = field(default_factory=list)

    def save(self, path: str):
        np.savez(path, f=self.f.cpu().numpy(), f_prev=self.f_prev.cpu().numpy(), v=self.v.cpu().numpy(),
                 alpha=self.alpha, k=self.k, history=np.array(self.history, dtype=np.float64))

    @staticmethod
    def load(path: str, device):
        d = np.load(path)
        t = lambda a: torch.from_numpy(a).to(device)  # noqa: E731
        return FistaState(t(d["f"]), t(d["f_prev"]), t(d["v"]), float(d["alpha"]), int(d["k"]),
                          [tuple(r) for r in d["history"]])


def fista(prob: Problem, f0: torch.Tensor, iters: int, gamma0: float, tau: float, tv_iters: int = 20,
          subset: int | None = None, seed: int = 0, batched: bool = True, state: FistaState | None = None,
          checkpoint: str | None = None, checkpoint_every: int = 0, f_true: torch.Tensor | None = None):
    """Runs `iters` FISTA iterations (Alg. 1); returns the final state (history: (k, loss, rel_err, s))."""
    rng = np.random.default_rng(seed)
    Q = prob.kvec.shape[0]
    st = state or FistaState(f0.clone(), f0.clone(), f0.clone())
    t0 = time.perf_counter()
    for _ in range(iters):
        views = None if not subset else sorted(rng.choice(Q, size=subset, replace=False).tolist())
        loss, d = data_grad(prob, st.v, views, batched)
        if views is not None:
            d = d * (Q / len(views))
        gamma = gamma0 / math.sqrt(st.k)
        f_new = prox_tv_nonneg(st.v - gamma * d, gamma * tau, tv_iters)
        alpha_next = (1.0 + math.sqrt(1.0 + 4.0 * st.alpha * st.alpha)) / 2.0
        st.v = f_new + ((st.alpha - 1.0) / alpha_next) * (f_new - st.f)
        st.f_prev, st.f = st.f, f_new
        st.alpha = alpha_next
        err = float("nan")
        if f_true is not None:
            err = float((st.f - f_true).pow(2).sum() / f_true.pow(2).sum())
        st.history.append((st.k, loss, err, time.perf_counter() - t0))
        st.k += 1
        if checkpoint and checkpoint_every and st.k % checkpoint_every == 0:
            st.save(checkpoint)
    return st
