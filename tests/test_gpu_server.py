"""Serving (ls_submit / ls_poll): continuous batching gives, for every request, the same result as
a standalone call, whether it runs alone or in a mix of grids and request kinds."""
import time

import numpy as np
import pytest

import phantoms as ph

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib

TOL = 1e-5


def _standalone(ls, torch, f, kvec, meas=None):
    nz, ny, nx = f.shape
    plan = ls.Plan((nz, ny, nx), KB, H, tol=1e-6)
    uin = plan.plane_waves(kvec)
    u, far, code, stats = plan.forward(f, uin)
    out = {"u": u, "far": far}
    if meas is not None:
        res = torch.empty_like(far)
        l2 = ls.ls_residual(far, meas, res)
        yy = [float(torch.vdot(m.flatten(), m.flatten()).real) for m in meas]
        w = [1.0 / v for v in yy]
        g, _, _ = plan.gradient(f, res, u_fwd=u, weights=w)
        out["grad"] = g
        out["loss"] = 0.5 * float(np.sum(l2 * np.array(w)))
    torch.cuda.synchronize()
    plan.close()
    return out


def _case(torch, shape, views, seed, with_meas):
    dn = ph.random_ellipsoids(shape, count=3, rmin=2, rmax=min(shape) // 4, dn_max=0.05, seed=seed)
    f = to_dev(torch, potential(dn), torch.float32)
    kvec = ph.cone_directions(views, 0.8) * KB
    meas = None
    if with_meas:
        meas = to_dev(torch, ph.complex_normal((views, shape[1], shape[2]), seed=seed + 1) * 1e-3, torch.complex64)
    return f, kvec, meas


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix():
    torch, ls = torch_and_lib()
    cases = [((24, 24, 24), 6, 11, False), ((16, 16, 16), 3, 12, True), ((24, 24, 24), 4, 13, True),
             ((32, 32, 32), 5, 14, False), ((16, 16, 16), 2, 15, False), ((32, 32, 32), 3, 16, True)]
    data = [_case(torch, *c) for c in cases]
    ref = [_standalone(ls, torch, f, k, m) for (f, k, m) in data]
    srv = ls.Server(KB, H, tol=1e-6)
    outs, tickets = [], []
    for i, ((shape, views, seed, grad), (f, k, m)) in enumerate(zip(cases, data)):
        u = torch.empty((views,) + shape, dtype=torch.complex64, device="cuda")
        far = torch.empty((views, shape[1], shape[2]), dtype=torch.complex64, device="cuda")
        g = torch.empty(shape, dtype=torch.float32, device="cuda") if grad else None
        if grad:
            t = srv.submit_gradient(f, k, m, g, u_out=u)
        else:
            t = srv.submit_forward(f, k, u_out=u, far=far)
        outs.append((u, far, g))
        tickets.append(t)
        if i == 2:
            time.sleep(0.05)   # later requests arrive while the first ones are on the GPU
    infos = []
    for t in tickets:
        code, info = srv.wait(t)
        assert code == ls.LS_OK, info
        infos.append(info)
    for (shape, views, seed, grad), (u, far, g), r, info in zip(cases, outs, ref, infos):
        assert rel(u.cpu().numpy(), r["u"].cpu().numpy()) < TOL
        if grad:
            assert rel(g.cpu().numpy(), r["grad"].cpu().numpy()) < TOL
            assert info["loss"] == pytest.approx(r["loss"], rel=1e-5)
        else:
            assert rel(far.cpu().numpy(), r["far"].cpu().numpy()) < TOL
        assert info["ms"] > 0 and info["iterations_max"] > 0
    srv.close()


@pytest.mark.gpu
def test_request_that_cannot_fit_is_refused_and_unknown_tickets_fail():
    torch, ls = torch_and_lib()
    srv = ls.Server(KB, H, hbm_budget_bytes=64 << 20)
    f = torch.zeros((64, 64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(ls.LsError) as e:
        srv.submit_forward(f, ph.cone_directions(8, 0.8) * KB)
    assert e.value.code == ls.LS_EAGAIN
    with pytest.raises(ls.LsError) as e:
        ls.ls_poll(srv.handle, 12345)
    assert e.value.code == ls.LS_ENOTFOUND
    srv.close()
