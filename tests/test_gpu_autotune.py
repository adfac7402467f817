"""Launch-variant autotuner: the variants it picks are valid, every variant gives the oracle's fields,
and its cache file round-trips."""
import os

import numpy as np
import pytest

import phantoms as ph

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib
from test_gpu_forward import TOL_FIELD, _oracle_views

SHAPE = (32, 32, 32)


def _setup(torch, ls, n_views):
    f64 = potential(ph.random_ellipsoids(SHAPE, count=4, rmin=3, rmax=8, dn_max=0.03))
    f = to_dev(torch, f64, torch.float32)
    k = ph.cone_directions(n_views, 0.8) * KB
    return f64, f, k


def _key(torch, n_views):
    nz, ny, nx = SHAPE
    return f"{torch.cuda.get_device_name().replace(' ', '_')}:{nx}x{ny}x{nz}:{n_views}"


@pytest.mark.gpu
def test_autotune_picks_valid_variants_and_keeps_the_results(monkeypatch):
    torch, ls = torch_and_lib()
    monkeypatch.delenv("LS_AUTOTUNE_CACHE", raising=False)
    f64, f, k = _setup(torch, ls, 4)
    ref = ls.Plan(SHAPE, KB, H, tol=1e-6)
    u_ref, far_ref, code, _ = ref.forward(f, ref.plane_waves(k))
    assert code == ls.LS_OK
    plan = ls.Plan(SHAPE, KB, H, tol=1e-6)
    t = plan.autotune(4, f)
    assert t["from_cache"] == 0
    assert t["z_tma"] in (0, 1) and t["ix_prefetch"] in (0, 1) and t["fx_views_fastest"] in (0, 1)
    assert t["check_every"] in (2, 4, 8) and t["use_graphs"] in (0, 1)
    assert t["z_split"] in (0, 1) and t["strided_wide"] in (0, 1) and t["views_per_launch"] in (0, 1, 2, 8)
    assert t["z_persist"] in (0, 1, 2) and t["fx_bulk"] in (0, 1)
    assert t["matvec_us_per_view"] > 0 and t["solve_ms"] > 0
    u, far, code, stats = plan.forward(f, plan.plane_waves(k))
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    for q in range(4):
        assert rel(u[q].cpu().numpy(), u_ref[q].cpu().numpy()) < TOL_FIELD
        assert rel(far[q].cpu().numpy(), far_ref[q].cpu().numpy()) < TOL_FIELD
    plan.close()
    ref.close()


# (z_tma, ix_prefetch, fx_views_fastest, check_every, use_graphs, z_split, strided_wide, views_per_launch,
#  z_persist, fx_bulk)
VARIANTS = [(0, 0, 0, 2, 0, 0, 0, 0, 0, 0), (1, 0, 1, 8, 1, 1, 1, 2, 0, 1), (0, 1, 0, 4, 1, 0, 1, 1, 0, 0),
            (1, 1, 0, 2, 1, 1, 0, 0, 1, 1), (1, 1, 1, 2, 0, 0, 1, 1, 1, 0), (1, 0, 0, 4, 1, 0, 0, 2, 1, 1),
            (1, 1, 0, 2, 1, 0, 0, 0, 2, 0), (1, 0, 1, 4, 0, 0, 1, 1, 2, 1)]
NAMES = ("z_tma", "ix_prefetch", "fx_views_fastest", "check_every", "use_graphs", "z_split", "strided_wide",
         "views_per_launch", "z_persist", "fx_bulk")


@pytest.mark.gpu
@pytest.mark.parametrize("variant", VARIANTS)
def test_every_variant_matches_the_oracle(tmp_path, monkeypatch, variant):
    # a cache entry forces the variant without timing anything
    torch, ls = torch_and_lib()
    n = 3
    cache = tmp_path / "tune.txt"
    v = [str(x) for x in variant]
    cache.write_text(_key(torch, n) + " " + " ".join(v[:5]) + " 1.0 1.0 " + " ".join(v[5:]) + "\n")
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(cache))
    f64, f, k = _setup(torch, ls, n)
    plan = ls.Plan(SHAPE, KB, H, tol=1e-6)
    t = plan.autotune(n, f)
    assert t["from_cache"] == 1
    assert tuple(t[k] for k in NAMES) == variant
    u, far, code, stats = plan.forward(f, plan.plane_waves(k))
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    for q, (_, u_o, far_o) in enumerate(_oracle_views(SHAPE, f64, k)):
        assert rel(u[q].cpu().numpy(), u_o) < TOL_FIELD
        assert rel(far[q].cpu().numpy(), far_o) < TOL_FIELD
    plan.close()


@pytest.mark.gpu
def test_cache_round_trip(tmp_path, monkeypatch):
    torch, ls = torch_and_lib()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(cache))
    _, f, _ = _setup(torch, ls, 2)
    plan = ls.Plan(SHAPE, KB, H, tol=1e-6)
    first = plan.autotune(2, f)
    assert first["from_cache"] == 0
    assert cache.read_text().split()[0] == _key(torch, 2)
    second = plan.autotune(2, f)
    assert second["from_cache"] == 1
    for name in NAMES:
        assert second[name] == first[name]
    assert np.isclose(second["solve_ms"], first["solve_ms"], rtol=1e-3)
    plan.close()
