"""torch.autograd bridge (checkpointed forward fields, ls_gradient backward) and FISTA/TV (Alg. 1)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import model

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib


def _setup(torch, ls, shape=(16, 16, 16), views=4, dn_max=0.05, seed=7):
    f_true64 = potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=min(shape) // 3, dn_max=dn_max,
                                              seed=seed))
    kvec = ph.cone_directions(views, 0.8) * KB
    plan = ls.Plan(shape, KB, H, tol=1e-7)
    f_true = to_dev(torch, f_true64, torch.float32)
    uin = plan.plane_waves(kvec)
    _, y, _, _ = plan.forward(f_true, uin, want_fields=False)
    return plan, kvec, uin, f_true, f_true64, y


@pytest.mark.gpu
def test_autograd_gradient_matches_ls_gradient_and_oracle():
    torch, ls = torch_and_lib()
    from paper_1910_13844_gb300.autograd import LSForward, data_loss

    plan, kvec, uin, f_true, f_true64, y = _setup(torch, ls)
    f0 = (0.9 * f_true).clone().requires_grad_(True)
    far = LSForward.apply(f0, plan, uin)
    loss = data_loss(far, y)
    loss.backward()
    g_auto = f0.grad.detach().clone()
    # direct library path with the same residual weighting
    u, far2, _, _ = plan.forward(f0.detach(), uin)
    res = torch.empty_like(far2)
    ls.ls_residual(far2, y, res)
    w = [1.0 / float(torch.vdot(m.flatten(), m.flatten()).real) for m in y]
    g_lib, _, _ = plan.gradient(f0.detach(), res, u_fwd=u, weights=w)
    torch.cuda.synchronize()
    assert rel(g_auto.cpu().numpy(), g_lib.cpu().numpy()) < 1e-5
    # oracle
    st = model.setup_from_optics(f0.shape, LAM, ETA_B, H)
    op = model.Operator(st)
    f064 = f0.detach().cpu().numpy().astype(np.float64)
    uins = [model.plane_wave(f0.shape, H, k) for k in kvec]
    ys = [yy.cpu().numpy().astype(np.complex128) for yy in y]
    g_ref = model.gradient(op, f064, uins, ys, tol=1e-12)
    assert rel(g_auto.cpu().numpy(), g_ref) < 1e-3
    plan.close()


@pytest.mark.gpu
def test_fista_tv_reduces_error_and_batched_equals_one_view_at_a_time(tmp_path):
    torch, ls = torch_and_lib()
    from paper_1910_13844_gb300 import recon

    plan, kvec, uin, f_true, f_true64, y = _setup(torch, ls, views=6)
    prob = recon.Problem(plan, kvec, y)
    f0 = torch.zeros_like(f_true)
    kw = dict(gamma0=2.0 / (KB * KB * 1e-3), tau=1e-4, tv_iters=10, f_true=f_true)
    # step size: scale of 1/(Lipschitz) estimated from the data term's curvature on this problem
    loss0, d0 = recon.data_grad(prob, f0)
    gamma0 = 0.5 * float(f_true.abs().max()) / float(d0.abs().max())
    kw["gamma0"] = gamma0
    a = recon.fista(prob, f0, 12, **kw)
    b = recon.fista(prob, f0, 12, batched=False, **kw)
    errs = [h[2] for h in a.history]
    losses = [h[1] for h in a.history]
    assert errs[-1] < errs[0] and errs[-1] < 0.7      # relative error from 1.0 at f = 0
    assert losses[-1] < 0.5 * losses[0]
    assert rel(a.f.cpu().numpy(), b.f.cpu().numpy()) < 1e-5
    # checkpoint / resume gives the same iterates as an uninterrupted run
    path = str(tmp_path / "fista.npz")
    c = recon.fista(prob, f0, 6, **kw)
    c.save(path)
    c2 = recon.fista(prob, f0, 6, state=recon.FistaState.load(path, f0.device), **kw)
    assert rel(c2.f.cpu().numpy(), a.f.cpu().numpy()) < 1e-5
    plan.close()
