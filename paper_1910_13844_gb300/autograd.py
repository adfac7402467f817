"""torch.autograd bridge to the LS forward model (eqs. lipp1, lipp2) and its adjoint gradient.

``LSForward.apply(f, plan, u_in)`` returns the far fields of all views (Q, my, mx).
Its backward calls ``ls_gradient`` with the forward fields saved by the forward
pass (checkpoint), so no forward solve is repeated.

For a real input f and complex output y = H(f), PyTorch hands backward the
conjugate-Wirtinger gradient g = dL/dRe(y) + i dL/dIm(y) and expects
dL/df = Re(J^H g).  With J = G~ (I - diag(f) G)^{-1} diag(u) this is
Re(conj(u) .* w), (I - G^H diag f) w = G~^H g, which is what ls_gradient
computes with unit view weights.
"""
from __future__ import annotations

import torch

from . import LS_BREAKDOWN, LsError, Plan


class LSForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: Plan, u_in: torch.Tensor) -> torch.Tensor:
        f = f.detach().contiguous()
        u, far, code, stats = plan.forward(f, u_in.contiguous(), want_fields=True, want_far=True)
        if code == LS_BREAKDOWN:
            raise LsError(code, "LSForward")
        ctx.plan = plan
        ctx.stats = stats
        ctx.save_for_backward(f, u)
        return far

    @staticmethod
    def backward(ctx, grad_far: torch.Tensor):
        f, u = ctx.saved_tensors
        g, code, stats = ctx.plan.gradient(f, grad_far.contiguous(), u_fwd=u)
        if code == LS_BREAKDOWN:
            raise LsError(code, "LSForward.backward")
        return g, None, None


def data_loss(far: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """sum_q ||far_q - y_q||^2 / (2 ||y_q||^2) (eq. prob)."""
    q = far.shape[0]
    diff = (far - y).reshape(q, -1)
    yn = y.reshape(q, -1).abs().pow(2).sum(dim=1)
    return 0.5 * (diff.abs().pow(2).sum(dim=1) / yn).sum()
