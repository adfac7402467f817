"""GPU forward model (batched BiCGStab + far field) vs the FP64 oracle (eqs. lipp1, lipp2)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import model

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib

TOL_FIELD = 1e-4   # relative L2 bound on total and far fields


def _oracle_views(shape, f64, kvecs, det=None):
    st = model.setup_from_optics(shape, LAM, ETA_B, H, m=det)
    op = model.Operator(st)
    out = []
    for k in kvecs:
        uin = model.plane_wave(shape, H, k)
        u = model.forward(op, f64, uin, tol=1e-12)
        out.append((uin, u, op.farfield_fft(f64 * u)))
    return out


@pytest.mark.gpu
def test_sphere_32_single_view_matches_oracle():
    # 32^3 grid, sphere of radius 10 voxels, dn = 0.02, plane wave along z, tol 1e-6
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f64 = potential(ph.sphere(shape, 10.0, 0.02))
    k = np.array([[0.0, 0.0, KB]])
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    f = to_dev(torch, f64, torch.float32)
    uin = plan.plane_waves(k)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    assert stats[0]["iterations"] > 0 and stats[0]["true_rel_residual"] <= 1e-5
    (uin_o, u_o, far_o), = _oracle_views(shape, f64, k)
    assert rel(uin[0].cpu().numpy(), uin_o) < 1e-6
    assert rel(u[0].cpu().numpy(), u_o) < TOL_FIELD
    assert rel(far[0].cpu().numpy(), far_o) < TOL_FIELD
    plan.close()


@pytest.mark.gpu
def test_zero_potential_returns_incident_field_exactly():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    plan = ls.Plan(shape, KB, H)
    f = torch.zeros(shape, dtype=torch.float32, device="cuda")
    uin = plan.plane_waves(ph.cone_directions(3, 0.8) * KB)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    assert torch.equal(u, uin)
    assert float(far.abs().max()) == 0.0
    assert all(s["iterations"] == 0 for s in stats)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,det", [((16, 24, 32), None), ((24, 16, 12), (12, 8))])
def test_batched_views_non_cubic_match_oracle(shape, det):
    torch, ls = torch_and_lib()
    f64 = potential(ph.random_ellipsoids(shape, count=6, rmin=2, rmax=min(shape) // 3, dn_max=0.05))
    kvecs = ph.cone_directions(5, 0.8) * KB
    opts = {"tol": 1e-6}
    if det is not None:
        opts.update(det_my=det[0], det_mx=det[1])
    plan = ls.Plan(shape, KB, H, **opts)
    f = to_dev(torch, f64, torch.float32)
    uin = plan.plane_waves(kvecs)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    ref = _oracle_views(shape, f64, kvecs, det)
    for q, (uin_o, u_o, far_o) in enumerate(ref):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
        assert rel(far[q].cpu().numpy(), far_o) < TOL_FIELD
    plan.close()


@pytest.mark.gpu
def test_graph_replay_equals_direct_launches_bitwise():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    f64 = potential(ph.sphere(shape, 5.0, 0.05))
    kvecs = ph.cone_directions(3, 0.8) * KB
    res = []
    for graphs in (1, 0):
        plan = ls.Plan(shape, KB, H, use_graphs=graphs)
        f = to_dev(torch, f64, torch.float32)
        uin = plan.plane_waves(kvecs)
        u, far, code, stats = plan.forward(f, uin)
        torch.cuda.synchronize()
        res.append((u.clone(), far.clone()))
        plan.close()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


@pytest.mark.gpu
def test_not_converged_status_is_reported():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    f64 = potential(ph.sphere(shape, 6.0, 0.1))
    plan = ls.Plan(shape, KB, H, max_iter=2, max_restarts=0)
    f = to_dev(torch, f64, torch.float32)
    uin = plan.plane_waves(np.array([[0.0, 0.0, KB]]))
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_NOT_CONVERGED
    assert stats[0]["iterations"] == 2
    plan.close()


@pytest.mark.gpu
def test_builtin_plane_waves_equal_explicit_incident_fields():
    # u_in == NULL: the plan's cone of plane waves (sin theta = NA / eta_b, phi_q = 2 pi q / Q), generated in
    # the solver's workspace; the same solve with the explicit fields, and the oracle's
    torch, ls = torch_and_lib()
    shape = (24, 32, 32)
    Q = 3
    f64 = potential(ph.random_ellipsoids(shape, count=3, rmin=2, rmax=6, seed=31))
    f = to_dev(torch, f64, torch.float32)
    plan = ls.Plan(shape, KB, H, tol=1e-6, cone_sin_theta=0.8 / ETA_B)
    kvec = ph.cone_directions(Q, 0.8) * KB
    u_ref, far_ref, code_ref, _ = plan.forward(f, plan.plane_waves(kvec))
    u, far, code, stats = plan.forward(f, None, n_views=Q)
    torch.cuda.synchronize()
    assert code == ls.LS_OK and code_ref == ls.LS_OK
    assert rel(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-6
    assert rel(far.cpu().numpy(), far_ref.cpu().numpy()) < 1e-6
    for q, (uin_o, u_o, far_o) in enumerate(_oracle_views(shape, f64, kvec)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
        assert rel(far[q].cpu().numpy(), far_o) < TOL_FIELD
    # the gradient recomputes its forward fields from the built-in waves when u_in and u_fwd are NULL
    res = far.clone()
    g_ref, _, _ = plan.gradient(f, res, u_fwd=u_ref)
    g, code, _ = plan.gradient(f, res)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    assert rel(g.cpu().numpy(), g_ref.cpu().numpy()) < 1e-5
    plan.close()
