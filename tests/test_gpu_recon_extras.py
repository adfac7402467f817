"""Reconstruction extras on the GPU: the fused FGP evaluation of prox_{lam TV + i_{>=0}} (Alg. 1 prox
step) against the FP64 oracle, and warm-started forward solves (ls_forward_warm)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import tv

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib


@pytest.mark.gpu
@pytest.mark.parametrize("shape,iters", [((24, 20, 16), 20), ((7, 5, 9), 50), ((128, 128, 128), 20)])
def test_prox_tv_matches_oracle(shape, iters):
    torch, ls = torch_and_lib()
    rng = np.random.default_rng(11)
    z = 0.5 + rng.standard_normal(shape)
    lam = 0.15
    zd = to_dev(torch, z, torch.float32)
    x = torch.empty_like(zd)
    ls.ls_prox_tv(zd, x, lam, iters)
    torch.cuda.synchronize()
    ref = tv.prox_tv_nonneg(zd.cpu().numpy().astype(np.float64), lam, iters)
    assert rel(x.cpu().numpy(), ref) < 1e-5
    assert float(x.min()) >= 0.0
    # caller-provided workspace gives the same bits
    work = torch.empty(6 * zd.numel(), dtype=torch.float32, device="cuda")
    x2 = torch.empty_like(zd)
    ls.ls_prox_tv(zd, x2, lam, iters, work=work)
    torch.cuda.synchronize()
    assert torch.equal(x, x2)


@pytest.mark.gpu
def test_prox_tv_edge_cases():
    torch, ls = torch_and_lib()
    z = to_dev(torch, np.random.default_rng(2).standard_normal((6, 5, 4)), torch.float32)
    x = torch.empty_like(z)
    ls.ls_prox_tv(z, x, 0.0, 10)          # lam = 0: projection on the orthant, exactly
    torch.cuda.synchronize()
    assert torch.equal(x, z.clamp_min(0.0))
    y = z.clone()
    ls.ls_prox_tv(y, y, -1.0, 5)          # in place allowed without TV
    torch.cuda.synchronize()
    assert torch.equal(y, z.clamp_min(0.0))
    with pytest.raises(ls.LsError) as e:  # z is read every iteration: no aliasing with lam > 0
        ls.ls_prox_tv(y, y, 0.1, 5)
    assert e.value.code == ls.LS_EINVAL
    one = to_dev(torch, np.array([[[-0.5]]]), torch.float32)   # a single voxel: TV = 0
    out = torch.empty_like(one)
    ls.ls_prox_tv(one, out, 0.3, 4)
    torch.cuda.synchronize()
    assert float(out) == 0.0


@pytest.mark.gpu
def test_warm_started_forward_solves():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=5, rmin=3, rmax=9, dn_max=0.05)), torch.float32)
    kvec = ph.cone_directions(4, 0.8) * KB
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    uin = plan.plane_waves(kvec)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    cold_iters = [s["iterations"] for s in stats]
    # from the converged fields: the initial true residual meets the tolerance (or one step does)
    u2 = plan.field(4)
    far2 = plan.detector(4)
    code2, st2 = ls.ls_forward_warm(plan.handle, f, uin, u, u2, far2)
    torch.cuda.synchronize()
    assert code2 == ls.LS_OK
    assert all(s["iterations"] <= 1 for s in st2)
    assert rel(u2.cpu().numpy(), u.cpu().numpy()) < 1e-6
    # from the fields of a slightly different potential, in place: fewer iterations, same solution
    u3, _, _, _ = plan.forward(1.05 * f, uin)
    code3, st3 = ls.ls_forward_warm(plan.handle, f, uin, u3, u3, far2)
    torch.cuda.synchronize()
    assert code3 == ls.LS_OK
    assert sum(s["iterations"] for s in st3) < sum(cold_iters)
    assert rel(u3.cpu().numpy(), u.cpu().numpy()) < 1e-5
    assert rel(far2.cpu().numpy(), far.cpu().numpy()) < 1e-5
    plan.close()


@pytest.mark.gpu
def test_fista_with_warm_starts_matches_cold_starts():
    torch, ls = torch_and_lib()
    from paper_1910_13844_gb300 import recon

    # a strong scatterer and a start near the solution: the potential changes little between
    # iterations, so each view's previous field is a good initial guess
    shape = (32, 32, 32)
    f_true = to_dev(torch, potential(ph.random_ellipsoids(shape, count=5, rmin=4, rmax=10, dn_max=0.1)),
                    torch.float32)
    kvec = ph.cone_directions(6, 0.8) * KB
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    uin = plan.plane_waves(kvec)
    _, y, code, _ = plan.forward(f_true, uin, want_fields=False)
    prob = recon.Problem(plan, kvec, y)
    f0 = 0.95 * f_true
    _, d0 = recon.data_grad(prob, torch.zeros_like(f_true))
    kw = dict(gamma0=0.5 * float(f_true.abs().max()) / float(d0.abs().max()), tau=1e-4, tv_iters=10)
    cold_stats, warm_stats = [], []
    a = recon.fista(prob, f0, 6, solver_stats=cold_stats, **kw)
    b = recon.fista(prob, f0, 6, warm_start=True, solver_stats=warm_stats, **kw)
    assert rel(b.f.cpu().numpy(), a.f.cpu().numpy()) < 1e-4
    assert sum(s["iterations"] for s in warm_stats) < sum(s["iterations"] for s in cold_stats)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,iters", [((12, 10, 9), 30), ((24, 20, 16), 20), ((64, 64, 64), 20), ((9, 1, 1), 40)])
def test_prox_hs_matches_oracle(shape, iters):
    from oracle import hessian as hs

    torch, ls = torch_and_lib()
    rng = np.random.default_rng(12)
    z = 0.5 + rng.standard_normal(shape)
    lam = 0.02
    zd = to_dev(torch, z, torch.float32)
    x = torch.empty_like(zd)
    ls.ls_prox_hs(zd, x, lam, iters)
    torch.cuda.synchronize()
    ref = hs.prox_hs_nonneg(zd.cpu().numpy().astype(np.float64), lam, iters)
    assert rel(x.cpu().numpy(), ref) < 1e-4
    assert float(x.min()) >= 0.0
    y = torch.empty_like(zd)
    ls.ls_prox_hs(zd, y, 0.0, 5)
    torch.cuda.synchronize()
    assert torch.equal(y, zd.clamp_min(0.0))
    with pytest.raises(ls.LsError):
        ls.ls_prox_hs(zd, zd, lam, 5)


@pytest.mark.gpu
def test_fista_with_the_hessian_schatten_regulariser_reduces_the_error():
    torch, ls = torch_and_lib()
    from paper_1910_13844_gb300 import recon

    shape = (32, 32, 32)
    f_true = to_dev(torch, potential(ph.random_ellipsoids(shape, count=5, rmin=4, rmax=10, dn_max=0.05)),
                    torch.float32)
    kvec = ph.cone_directions(8, 0.8) * KB
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    uin = plan.plane_waves(kvec)
    _, y, code, _ = plan.forward(f_true, uin, want_fields=False)
    prob = recon.Problem(plan, kvec, y)
    f0 = torch.zeros_like(f_true)
    _, d0 = recon.data_grad(prob, f0)
    kw = dict(gamma0=0.5 * float(f_true.abs().max()) / float(d0.abs().max()), tau=1e-5, tv_iters=10,
              f_true=f_true)
    st = recon.fista(prob, f0, 10, reg="hs", **kw)
    errs = [h[2] for h in st.history]
    assert errs[-1] < errs[0] and errs[-1] < 0.9      # squared relative error from 1.0 at f = 0
    assert float(st.f.min()) >= 0.0
    plan.close()
