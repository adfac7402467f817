"""Edge cases of the GPU path: empty batches, zero incident fields, the largest batch a call accepts,
and views of very different difficulty solved in one batch (per-view convergence masks)."""
import numpy as np
import pytest

import phantoms as ph

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib

MAX_VIEWS = 1024   # views per call (slot tables are sized by it)


@pytest.mark.gpu
def test_empty_batches_are_argument_errors():
    torch, ls = torch_and_lib()
    shape = (8, 8, 8)
    plan = ls.Plan(shape, KB, H)
    f = torch.zeros(shape, dtype=torch.float32, device="cuda")
    none = plan.field(0)
    for call in (lambda: ls.ls_forward(plan.handle, f, none, none),
                 lambda: ls.ls_matvec_batch(plan.handle, f, none, none),
                 lambda: ls.ls_plane_waves(plan.handle, np.zeros((0, 3)), none)):
        with pytest.raises(ls.LsError) as e:
            call()
        assert e.value.code == ls.LS_EINVAL
    plan.close()


@pytest.mark.gpu
def test_zero_incident_field_gives_zero_fields_without_iterating():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    f = to_dev(torch, potential(ph.sphere(shape, 5.0, 0.05)), torch.float32)
    plan = ls.Plan(shape, KB, H)
    uin = torch.zeros((2,) + shape, dtype=torch.complex64, device="cuda")
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    assert all(s["iterations"] == 0 for s in stats)
    assert float(u.abs().max()) == 0.0 and float(far.abs().max()) == 0.0
    plan.close()


@pytest.mark.gpu
def test_largest_batch_matches_single_view_solves():
    torch, ls = torch_and_lib()
    shape = (8, 8, 8)
    f = to_dev(torch, potential(ph.sphere(shape, 3.0, 0.05)), torch.float32)
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    kvec = ph.cone_directions(MAX_VIEWS, 0.8) * KB
    uin = plan.plane_waves(kvec)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK and len(stats) == MAX_VIEWS
    for q in (0, 511, MAX_VIEWS - 1):
        u1, far1, c1, _ = plan.forward(f, uin[q:q + 1].clone())
        torch.cuda.synchronize()
        assert c1 == ls.LS_OK
        assert rel(u[q].cpu().numpy(), u1[0].cpu().numpy()) < 1e-5
        assert rel(far[q].cpu().numpy(), far1[0].cpu().numpy()) < 1e-5
    big = torch.zeros((MAX_VIEWS + 1,) + shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(ls.LsError) as e:
        plan.forward(f, big)
    assert e.value.code == ls.LS_EINVAL
    plan.close()


@pytest.mark.gpu
def test_views_of_different_difficulty_in_one_batch():
    # a zero field (done at once), a weak and a strong illumination of one direction, and a third
    # direction: each view's result equals its own solve, whatever the others do
    torch, ls = torch_and_lib()
    shape = (24, 24, 24)
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=4, rmin=3, rmax=7, dn_max=0.1)), torch.float32)
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    k = ph.cone_directions(4, 0.8) * KB
    k[2] = k[1]                      # views 1 and 2: one direction, amplitudes 1e-3 and 1e3
    uin = plan.plane_waves(k)
    uin[0].zero_()
    uin[1] *= 1e-3
    uin[2] *= 1e3
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    assert stats[0]["iterations"] == 0 and stats[3]["iterations"] > 0
    for q in range(1, 4):
        u1, far1, c1, _ = plan.forward(f, uin[q:q + 1].clone())
        torch.cuda.synchronize()
        assert rel(u[q].cpu().numpy(), u1[0].cpu().numpy()) < 1e-5
    # linearity in the incident field survives the per-view scaling
    assert rel((u[1] * 1e6).cpu().numpy(), u[2].cpu().numpy()) < 1e-4
    plan.close()
