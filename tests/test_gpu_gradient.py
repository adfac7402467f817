"""GPU far-field operators and data-fidelity gradient vs the FP64 oracle (eq. Gtild-1, Alg. 1 line 6)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import model

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib


@pytest.mark.gpu
@pytest.mark.parametrize("shape,det", [((16, 16, 16), None), ((12, 24, 16), (20, 12))])
def test_farfield_and_adjoint_match_oracle(shape, det):
    torch, ls = torch_and_lib()
    opts = {} if det is None else {"det_my": det[0], "det_mx": det[1]}
    plan = ls.Plan(shape, KB, H, **opts)
    st = model.setup_from_optics(shape, LAM, ETA_B, H, m=det)
    op = model.Operator(st)
    f64 = potential(ph.random_ellipsoids(shape, count=3, rmin=2, rmax=5))
    u = [ph.random_field(shape, 30 + q) for q in range(2)]
    f = to_dev(torch, f64, torch.float32)
    ud = torch.stack([to_dev(torch, x, torch.complex64) for x in u])
    far = plan.detector(2)
    ls.ls_farfield(plan.handle, f, ud, far)
    torch.cuda.synchronize()
    for q in range(2):
        ref = op.farfield_direct(f64 * ud[q].cpu().numpy().astype(np.complex128))
        assert rel(far[q].cpu().numpy(), ref) < 1e-5
    r = [ph.random_field(plan.det, 40 + q) for q in range(2)]
    rd = torch.stack([to_dev(torch, x, torch.complex64) for x in r])
    out = plan.field(2)
    ls.ls_farfield_adjoint(plan.handle, rd, out)
    torch.cuda.synchronize()
    for q in range(2):
        ref = op.farfield_adjoint_fft(rd[q].cpu().numpy().astype(np.complex128))
        assert rel(out[q].cpu().numpy(), ref) < 1e-5
    plan.close()


def _problem(shape, nviews):
    f_true = potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=min(shape) // 3, dn_max=0.05))
    kvecs = ph.cone_directions(nviews, 0.8) * KB
    st = model.setup_from_optics(shape, LAM, ETA_B, H)
    op = model.Operator(st)
    ys = []
    for q, k in enumerate(kvecs):
        u = model.forward(op, f_true, model.plane_wave(shape, H, k), tol=1e-12)
        y = op.farfield_fft(f_true * u)
        noise = ph.complex_normal(st.det, 13845 + q)
        ys.append(y + 0.01 * np.linalg.norm(y) / np.sqrt(2 * y.size) * noise)
    return f_true, kvecs, op, ys


@pytest.mark.gpu
def test_gradient_matches_oracle():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    f_true, kvecs, op, ys = _problem(shape, 3)
    f0 = 0.9 * f_true
    plan = ls.Plan(shape, KB, H, tol=1e-7)
    f = to_dev(torch, f0, torch.float32)
    uin = plan.plane_waves(kvecs)
    u, far, code, _ = plan.forward(f, uin)
    y = torch.stack([to_dev(torch, x, torch.complex64) for x in ys])
    res = torch.empty_like(far)
    loss = ls.ls_residual(far, y, res)
    weights = [1.0 / float(np.vdot(x, x).real) for x in ys]
    g, code, stats = plan.gradient(f, res, u_fwd=u, weights=weights)
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    f032 = f.cpu().numpy().astype(np.float64)
    uins = [model.plane_wave(shape, H, k) for k in kvecs]
    g_ref = model.gradient(op, f032, uins, ys, tol=1e-12)
    assert rel(g.cpu().numpy(), g_ref) < 1e-3
    # the loss returned with the residuals is the oracle's data term
    L_ref = model.loss(op, f032, uins, ys, tol=1e-12)
    assert float(np.sum(loss * np.array(weights)) / 2) == pytest.approx(L_ref, rel=1e-4)
    # recomputing the forward fields inside ls_gradient gives the same gradient
    g2, code2, _ = plan.gradient(f, res, u_in=uin, weights=weights)
    torch.cuda.synchronize()
    assert rel(g2.cpu().numpy(), g.cpu().numpy()) < 1e-5
    plan.close()


@pytest.mark.gpu
def test_gradient_matches_central_differences():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    f_true, kvecs, op, ys = _problem(shape, 2)
    f0 = 0.9 * f_true
    plan = ls.Plan(shape, KB, H, tol=1e-7)
    y = torch.stack([to_dev(torch, x, torch.complex64) for x in ys])
    weights = [1.0 / float(np.vdot(x, x).real) for x in ys]

    def loss_and_grad(fnp, want_grad):
        f = to_dev(torch, fnp, torch.float32)
        uin = plan.plane_waves(kvecs)
        u, far, code, _ = plan.forward(f, uin)
        res = torch.empty_like(far)
        l2 = ls.ls_residual(far, y, res)
        L = 0.5 * float(np.sum(l2 * np.array(weights)))
        if not want_grad:
            return L, None
        g, _, _ = plan.gradient(f, res, u_fwd=u, weights=weights)
        torch.cuda.synchronize()
        return L, g.cpu().numpy().astype(np.float64)

    _, g = loss_and_grad(f0, True)
    rng = np.random.default_rng(3)
    d = rng.uniform(-1, 1, shape) * (f_true > 0)
    eps = 1e-3 * np.max(np.abs(f_true))   # the step of the central difference (1e-3 of max |f|)
    Lp, _ = loss_and_grad(f0 + eps * d, False)
    Lm, _ = loss_and_grad(f0 - eps * d, False)
    fd = (Lp - Lm) / (2 * eps)
    assert np.sum(g * d) == pytest.approx(fd, rel=2e-2)
    plan.close()
