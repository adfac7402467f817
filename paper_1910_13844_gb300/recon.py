"""Variational reconstruction on top of the LS model (Sec. 4, Alg. 1).

    f* in argmin_f  sum_q ||H_q(f) - y_q||^2 / (2 ||y_q||^2) + tau TV(f) + i_{>=0}(f)   (eq. prob)

solved by accelerated forward-backward splitting (FISTA, Alg. 1) with step
gamma_k = gamma_0 / sqrt(k), optional random view subsets per iteration
(Alg. 1 line 5), and the proximal operator of gamma tau TV + i_{>=0} evaluated
by the fast gradient projection method (FGP) on the dual of isotropic TV.
The data-term gradient (Alg. 1 line 6) comes from the CUDA library, batched
over the selected views (or one view per call, for comparison), with the forward
solves optionally warm-started from the previous iteration's fields; the TV prox
is the library's fused FGP kernels; the FISTA updates are element-wise tensor
operations on the device.

Reading of Alg. 1: the gradient is evaluated at the extrapolated point v^k
(standard FISTA), where the listing writes f^k.
"""
from __future__ import annotations

import json
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ls_forward, ls_forward_warm, ls_gradient, ls_plane_waves, ls_prox_hs, ls_prox_tv, ls_residual


# ------------------------------------------------------------------ TV prox (FGP)
def prox_tv_nonneg(z: torch.Tensor, lam: float, iters: int = 20) -> torch.Tensor:
    """argmin_x 0.5 ||x - z||^2 + lam TV(x) + i_{>=0}(x) by FGP (Beck and Teboulle 2009), in the library."""
    x = torch.empty_like(z)
    ls_prox_tv(z.contiguous(), x, lam, iters)
    return x


def prox_hs_nonneg(z: torch.Tensor, lam: float, iters: int = 20) -> torch.Tensor:
    """argmin_x 0.5 ||x - z||^2 + lam sum_v ||H x (v)||_{S1} + i_{>=0}(x) (Hessian Schatten norm), FGP."""
    x = torch.empty_like(z)
    ls_prox_hs(z.contiguous(), x, lam, iters)
    return x


PROX = {"tv": prox_tv_nonneg, "hs": prox_hs_nonneg}


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


def data_grad(prob: Problem, f: torch.Tensor, views=None, batched: bool = True, warm: dict | None = None,
              stats: list | None = None):
    """(loss, gradient) of the data term over `views` (all if None): batched, or one view per call.

    warm: a dict view -> field kept across calls; views found there start BiCGStab from that field
    (ls_forward_warm) and every view's new field is stored back.  stats: list that receives the
    per-view solver statistics of the forward solves."""
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
        if warm is not None and all(q in warm for q in g):
            for i, q in enumerate(g):
                u[i].copy_(warm[q])
            _, st = ls_forward_warm(plan.handle, f, uin, u, u, far)
        else:
            _, st = ls_forward(plan.handle, f, uin, u, far)
        if stats is not None:
            stats.extend(st)
        if warm is not None:
            for i, q in enumerate(g):
                warm[q] = u[i].clone()
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
    rng: dict | None = None      # state of the generator that draws the view subsets (numpy bit generator)

    def save(self, path: str):
        np.savez(path, f=self.f.cpu().numpy(), f_prev=self.f_prev.cpu().numpy(), v=self.v.cpu().numpy(),
                 alpha=self.alpha, k=self.k, history=np.array(self.history, dtype=np.float64),
                 rng=json.dumps(self.rng) if self.rng is not None else "")

    @staticmethod
    def load(path: str, device):
        d = np.load(path)
        t = lambda a: torch.from_numpy(a).to(device)  # noqa: E731
        rng = str(d["rng"]) if "rng" in d.files else ""
        return FistaState(t(d["f"]), t(d["f_prev"]), t(d["v"]), float(d["alpha"]), int(d["k"]),
                          [tuple(r) for r in d["history"]], json.loads(rng) if rng else None)


def fista(prob: Problem, f0: torch.Tensor, iters: int, gamma0: float, tau: float, tv_iters: int = 20,
          subset: int | None = None, seed: int = 0, batched: bool = True, state: FistaState | None = None,
          checkpoint: str | None = None, checkpoint_every: int = 0, f_true: torch.Tensor | None = None,
          warm_start: bool = False, solver_stats: list | None = None, reg: str = "tv"):
    """Runs `iters` FISTA iterations (Alg. 1); returns the final state (history: (k, loss, rel_err, s)).

    warm_start: start each view's forward solve from its field of the last iteration that used it.
    solver_stats: list that receives the forward solves' per-view statistics.
    reg: "tv" (total variation) or "hs" (Hessian Schatten 1-norm), both with positivity.
    A resumed run (state from a checkpoint) continues the view-subset draws where the saved run stopped."""
    prox = PROX[reg]
    rng = np.random.default_rng(seed)
    Q = prob.kvec.shape[0]
    st = state or FistaState(f0.clone(), f0.clone(), f0.clone())
    if st.rng is not None:
        rng.bit_generator.state = st.rng
    warm = {} if warm_start else None
    t0 = time.perf_counter()
    for _ in range(iters):
        views = None if not subset else sorted(rng.choice(Q, size=subset, replace=False).tolist())
        loss, d = data_grad(prob, st.v, views, batched, warm=warm, stats=solver_stats)
        if views is not None:
            d = d * (Q / len(views))
        gamma = gamma0 / math.sqrt(st.k)
        f_new = prox(st.v - gamma * d, gamma * tau, tv_iters)
        alpha_next = (1.0 + math.sqrt(1.0 + 4.0 * st.alpha * st.alpha)) / 2.0
        st.v = f_new + ((st.alpha - 1.0) / alpha_next) * (f_new - st.f)
        st.f_prev, st.f = st.f, f_new
        st.alpha = alpha_next
        err = float("nan")
        if f_true is not None:
            err = float((st.f - f_true).pow(2).sum() / f_true.pow(2).sum())
        st.history.append((st.k, loss, err, time.perf_counter() - t0))
        st.k += 1
        st.rng = rng.bit_generator.state
        if checkpoint and checkpoint_every and st.k % checkpoint_every == 0:
            st.save(checkpoint)
    return st
