"""Scattering potential on the GPU (Sec. 2.1) against the oracle, and the per-launch profiler's counts
against the solver's own statistics."""
import numpy as np
import pytest

import phantoms as ph
from oracle import green

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib


@pytest.mark.gpu
def test_scattering_potential_matches_oracle():
    torch, ls = torch_and_lib()
    dn = ph.random_ellipsoids((24, 20, 16), count=6, rmin=2, rmax=6, dn_max=0.1)
    dnd = to_dev(torch, dn, torch.float32)
    f = torch.empty_like(dnd)
    ls.ls_scattering_potential(dnd, ETA_B, KB, f)
    torch.cuda.synchronize()
    ref = green.scattering_potential(dnd.cpu().numpy().astype(np.float64), ETA_B, LAM)
    assert rel(f.cpu().numpy(), ref) < 1e-6
    assert float(f[dnd == 0].abs().max()) == 0.0


@pytest.mark.gpu
def test_profiler_counts_match_the_solver_statistics():
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=4, rmin=3, rmax=8, dn_max=0.05)), torch.float32)
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    uin = plan.plane_waves(ph.cone_directions(5, 0.8) * KB)
    ls.ls_profile(plan.handle, True)
    u, far, code, stats = plan.forward(f, uin)
    torch.cuda.synchronize()
    prof = ls.ls_profile(plan.handle, False)
    assert code == ls.LS_OK
    # every operator application runs each of the five passes once per view that is still running
    matvecs = sum(s["matvecs"] for s in stats)
    for kind in ("fx", "fy", "z", "iy", "ix"):
        ms, launches, slot_passes, active = prof[kind]
        assert ms > 0 and launches > 0
        assert active == matvecs, (kind, active, matvecs)
        assert slot_passes >= active
    assert prof["update"][3] == sum(s["iterations"] for s in stats)
    assert prof["far"][1] > 0
    plan.close()
