"""ls_matvec_noalloc, the operator for callers that cannot allocate device memory.

Some callers may not call cudaMalloc: a process whose device memory is all
owned by its own pool, or a loop that must not stall on the device
synchronisation an allocation can cause.  ls_matvec_noalloc applies the same
operator as ls_matvec using a static scratch array inside the library instead
of plan workspace.  This file is collected last on purpose.
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
    plan = ls.Plan(shape, KB, H)
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=6)), torch.float32)
    outs = []
    for call, adjoint in enumerate((False, True)):
        x = to_dev(torch, ph.random_field(shape, 100 + call), torch.complex64)
        ref = torch.empty_like(x)
        got = torch.full_like(x, float("nan"))
        ls.ls_matvec(plan.handle, f, x, ref, adjoint)
        ls.ls_matvec_noalloc(plan.handle, f, x, got, adjoint)
        torch.cuda.synchronize()
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) < TOL
        outs.append(got.cpu().numpy())
    # the second call does not see the first call's scratch contents
    assert rel(outs[1], outs[0]) > 0.1
    plan.close()


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
