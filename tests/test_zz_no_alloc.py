"""ls_matvec_noalloc, the operator for callers that cannot allocate device memory.

Some callers may not call cudaMalloc: a process whose device memory is all
owned by its own pool, or a loop that must not stall on the device
synchronisation an allocation can cause.  ls_matvec_noalloc applies the same
operator as ls_matvec using a static scratch array inside the library (reserved
when a plan is created) instead of plan workspace.  This file is collected last
on purpose.
"""
import numpy as np
import pytest

import phantoms as ph

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib

TOL = 1e-5   # the operator tests' relative L2 bound


@pytest.mark.gpu
def test_noalloc_matvec_matches_matvec_on_two_calls_in_a_row():
    torch, ls = torch_and_lib()
    shape = (24, 32, 48)   # (nz, ny, nx); ragged tiles along x
    big = (96, 96, 96)     # fills the static array with data of another layout first
    plan = ls.Plan(shape, KB, H)       # never runs ls_matvec: it has no workspace
    plan_big = ls.Plan(big, KB, H)
    ref_plan = ls.Plan(shape, KB, H)   # the existing entry point runs on a plan of its own
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=6)), torch.float32)
    f_big = to_dev(torch, potential(ph.random_ellipsoids(big, count=4, rmin=4, rmax=12, seed=3)), torch.float32)
    xs = [to_dev(torch, ph.random_field(shape, 100 + c), torch.complex64) for c in range(2)]
    x_big = to_dev(torch, ph.random_field(big, 99), torch.complex64)
    y_big = torch.empty_like(x_big)
    gots = [torch.full_like(x, float("nan")) for x in xs]
    refs = [torch.empty_like(x) for x in xs]
    # warm-up on both grids (the kernels' first launches), the larger grid last
    ls.ls_matvec_noalloc(plan.handle, f, xs[0], gots[0])
    ls.ls_matvec_noalloc(plan_big.handle, f_big, x_big, y_big)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for c, adjoint in enumerate((False, True)):
        gots[c].fill_(float("nan"))
        torch.cuda.synchronize()
        ls.ls_matvec_noalloc(plan.handle, f, xs[c], gots[c], adjoint)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0   # the call allocated nothing
    for c, adjoint in enumerate((False, True)):
        ls.ls_matvec(ref_plan.handle, f, xs[c], refs[c], adjoint)
    torch.cuda.synchronize()
    for c in range(2):
        got = gots[c].cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, refs[c].cpu().numpy()) < TOL
    for p in (plan, plan_big, ref_plan):
        p.close()


@pytest.mark.gpu
def test_noalloc_rejects_grids_beyond_the_static_scratch():
    torch, ls = torch_and_lib()
    shape = (128, 128, 128)   # needs 96 MiB of scratch, more than the 64 MiB array
    plan = ls.Plan(shape, KB, H)
    f = torch.zeros(shape, dtype=torch.float32, device="cuda")
    x = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(ls.LsError) as err:
        ls.ls_matvec_noalloc(plan.handle, f, x, y)
    assert err.value.code == ls.LS_EINVAL
    assert "static scratch" in str(err.value)
    plan.close()
