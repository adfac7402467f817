"""Failure paths of the solver and the server, made on purpose without faulting the GPU.

Each case is switched on with ls_debug_inject (test-only failure injection):
  * a zero shadow residual forces a BiCGStab breakdown (<rh, v> = 0 in the first iteration):
    LS_BREAKDOWN with no restarts allowed, recovery through a restart otherwise;
  * a host loop limited to a few rounds leaves views unfinished: LS_TIMEOUT;
  * failed workspace allocations give LS_ENOMEM, for a plan and for a server lane, and both stay
    usable afterwards;
  * the TMA-staged z pass waits on a barrier that nothing completes and gives up after a short
    limit (every copy it issued is still waited for): the solve returns LS_ECUDA, and the next solve
    on the same plan is correct.
Results after recovery are checked against the FP64 oracle.
"""
import numpy as np
import pytest

import phantoms as ph
from oracle import model

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib

TOL_FIELD = 1e-4


def _problem(torch, shape=(32, 32, 32), views=3, seed=7):
    f64 = potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=8, dn_max=0.05, seed=seed))
    kvec = ph.cone_directions(views, 0.8) * KB
    return f64, to_dev(torch, f64, torch.float32), kvec


def _oracle_fields(shape, f64, kvec):
    op = model.Operator(model.setup_from_optics(shape, LAM, ETA_B, H))
    return [model.forward(op, f64, model.plane_wave(shape, H, k), tol=1e-12) for k in kvec]


@pytest.mark.gpu
def test_zero_shadow_residual_breaks_down_without_restarts():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f64, f, kvec = _problem(torch, shape)
    plan = ls.Plan(shape, KB, H, tol=1e-6, max_restarts=0)
    uin = plan.plane_waves(kvec)
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_ZERO_SHADOW, 1)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_BREAKDOWN
    assert stats[1]["status"] == ls.LS_BREAKDOWN and stats[1]["restarts"] == 0
    assert stats[0]["status"] == ls.LS_OK and stats[2]["status"] == ls.LS_OK
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_NONE)
    plan.close()


@pytest.mark.gpu
def test_zero_shadow_residual_recovers_through_a_restart():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f64, f, kvec = _problem(torch, shape)
    plan = ls.Plan(shape, KB, H, tol=1e-6)   # default: up to 4 restarts from the true residual
    uin = plan.plane_waves(kvec)
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_ZERO_SHADOW, 1)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    assert stats[1]["restarts"] >= 1
    for q, u_o in enumerate(_oracle_fields(shape, f64, kvec)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_NONE)
    plan.close()


@pytest.mark.gpu
def test_bounded_host_loop_reports_timeout():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f64, f, kvec = _problem(torch, shape)
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    uin = plan.plane_waves(kvec)
    for rounds in (0, 2):
        ls.ls_debug_inject(plan.handle, ls.LS_INJECT_MAX_ROUNDS, rounds)
        _, _, code, stats = plan.forward(f, uin)
        torch.cuda.synchronize()
        assert code == ls.LS_TIMEOUT, rounds
        assert all(s["status"] == ls.LS_TIMEOUT for s in stats)
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_MAX_ROUNDS, -1)
    u, _, code, _ = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    for q, u_o in enumerate(_oracle_fields(shape, f64, kvec)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
    plan.close()


@pytest.mark.gpu
def test_failed_workspace_allocation_gives_enomem_and_the_plan_recovers():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f64, f, kvec = _problem(torch, shape)
    other = ls.Plan(shape, KB, H)
    uin3 = other.plane_waves(kvec)            # incident fields made outside the plan under test
    torch.cuda.synchronize()
    other.close()
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    _, _, code, _ = plan.forward(f, uin3[:1])  # workspace for one view
    assert code == ls.LS_OK
    ls.ls_debug_inject(None, ls.LS_INJECT_ALLOC_FAIL, 1)
    with pytest.raises(ls.LsError) as err:    # three views need a larger workspace: its allocation fails
        plan.forward(f, uin3)
    assert err.value.code == ls.LS_ENOMEM
    u, _, code, _ = plan.forward(f, uin3)     # the next allocation succeeds
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    for q, u_o in enumerate(_oracle_fields(shape, f64, kvec)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
    plan.close()


@pytest.mark.gpu
def test_failed_lane_allocation_gives_enomem_and_the_server_stays_usable():
    torch, ls = torch_and_lib()
    shape = (24, 24, 24)
    f64, f, kvec = _problem(torch, shape, views=2, seed=9)
    srv = ls.Server(KB, H, tol=1e-6)
    far1 = torch.empty((2,) + shape[1:], dtype=torch.complex64, device="cuda")
    far2 = torch.empty_like(far1)
    ls.ls_debug_inject(None, ls.LS_INJECT_ALLOC_FAIL, 1)   # the first lane's workspace
    code, _ = srv.wait(srv.submit_forward(f, kvec, far=far1))
    assert code == ls.LS_ENOMEM
    code, _ = srv.wait(srv.submit_forward(f, kvec, far=far2))
    assert code == ls.LS_OK
    torch.cuda.synchronize()
    op = model.Operator(model.setup_from_optics(shape, LAM, ETA_B, H))
    for q, u_o in enumerate(_oracle_fields(shape, f64, kvec)):
        assert rel(far2[q].cpu().numpy(), op.farfield_fft(f64 * u_o)) < TOL_FIELD
    srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("z_persist", [0, 2])
def test_z_pass_wait_that_runs_out_returns_ecuda_and_the_plan_stays_usable(tmp_path, monkeypatch, z_persist):
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)   # 64-point z transforms: the TMA-staged z pass
    f64, f, kvec = _problem(torch, shape)
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    if z_persist:
        # the dynamically scheduled form, forced through an autotune cache entry (default variants otherwise)
        nz, ny, nx = shape
        key = torch.cuda.get_device_name().replace(" ", "_") + f":{nx}x{ny}x{nz}:{len(kvec)}"
        cache = tmp_path / "tune.txt"
        cache.write_text(key + f" 1 1 0 2 1 1.0 1.0 0 0 0 {z_persist} 0\n")
        monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(cache))
        assert plan.autotune(len(kvec), f)["z_persist"] == z_persist
    uin = plan.plane_waves(kvec)
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_Z_STALL, 2_000_000)   # give up after 2 ms
    with pytest.raises(ls.LsError) as err:
        plan.forward(f, uin)
    assert err.value.code == ls.LS_ECUDA
    assert "TMA" in str(err.value)
    ls.ls_debug_inject(plan.handle, ls.LS_INJECT_NONE)
    u, far, code, _ = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    for q, u_o in enumerate(_oracle_fields(shape, f64, kvec)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
    plan.close()
