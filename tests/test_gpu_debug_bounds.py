"""The index-checking build (libls_debug.so, compiled with LS_DEBUG_BOUNDS): on the launch variants
of the hot path (TMA z pass in its default, second-split, persistent and dynamically scheduled forms, the column-group z
pass of the bead lengths, 16/32-pencil strided passes, the bulk-staged first pass, chunked
iterations) no index check fails and the results still match the FP64 oracle; a probe that makes
the first pass's slot check exclude one view shows that a failed check is recorded and the access
skipped, without a fault.  Runs in a child process (the debug library is chosen at import)."""
import os
import subprocess
import sys
import textwrap

import pytest

from gpu_common import torch_and_lib

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r'''
import json, os, sys
import numpy as np
import torch
sys.path.insert(0, os.path.join(os.environ["LS_ROOT"], "tests"))
import paper_1910_13844_gb300 as ls
import phantoms as ph
from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev
from oracle import model

assert ls.library_path().endswith("libls_debug.so"), ls.library_path()
checked, site = ls.ls_debug_bounds(clear=True)
assert checked and site == 0, (checked, site)

def oracle(shape, f64, kvec):
    op = model.Operator(model.setup_from_optics(shape, LAM, ETA_B, H))
    out = []
    for k in kvec:
        u = model.forward(op, f64, model.plane_wave(shape, H, k), tol=1e-12)
        out.append((u, op.farfield_fft(f64 * u)))
    return out

def case(name, shape, views, cache_line=None):
    f64 = potential(ph.random_ellipsoids(shape, count=3, rmin=2, rmax=6, dn_max=0.04, seed=3))
    f = to_dev(torch, f64, torch.float32)
    kvec = ph.cone_directions(views, 0.8) * KB
    plan = ls.Plan(shape, KB, H, tol=1e-6)
    if cache_line is not None:
        t = plan.autotune(views, f)
        assert t["from_cache"] == 1, t
    u, far, code, stats = plan.forward(f, plan.plane_waves(kvec))
    torch.cuda.synchronize()
    assert code == ls.LS_OK, (name, stats)
    worst = 0.0
    for q, (u_o, far_o) in enumerate(oracle(shape, f64, kvec)):
        worst = max(worst, rel(u[q].cpu().numpy(), u_o), rel(far[q].cpu().numpy(), far_o))
    assert worst < 1e-4, (name, worst)
    # the adjoint path: gradient of the data term at the forward fields
    g, code, _ = plan.gradient(f, far.clone(), u_fwd=u)
    torch.cuda.synchronize()
    assert code == ls.LS_OK and bool(torch.isfinite(g).all()), name
    plan.close()
    checked, site = ls.ls_debug_bounds(clear=True)
    assert checked and site == 0, (name, hex(site))
    print(name, "ok", worst, flush=True)

shape = (32, 32, 32)
case("defaults", shape, 3)
# every non-default launch variant at once, forced through an autotune cache entry
nz, ny, nx = shape
key = torch.cuda.get_device_name().replace(" ", "_") + f":{nx}x{ny}x{nz}:4"
open(os.environ["LS_AUTOTUNE_CACHE"], "w").write(key + " 1 1 1 2 1 1.0 1.0 1 1 2 1 1\n")
case("variants", shape, 4, cache_line=True)
# the dynamically scheduled z pass
open(os.environ["LS_AUTOTUNE_CACHE"], "w").write(key + " 1 1 0 2 1 1.0 1.0 0 0 0 2 0\n")
case("dynamic z", shape, 4, cache_line=True)
os.environ.pop("LS_AUTOTUNE_CACHE")
case("bead length 144", (72, 16, 16), 2)
# z lengths whose threads do several stage-2 sub-transforms (128: 16 x 8 on 8 threads, 192: 24 x 8 on
# 8, 384: 32 x 12 on 16), in the form untuned plans run for them
case("z length 128", (64, 16, 16), 2)
case("z length 192", (96, 16, 16), 2)
case("z length 384", (192, 16, 16), 2)
case("non-cubic", (24, 16, 32), 2)

# a failed check: the first pass's slot check excludes the last view of the launch
f64 = potential(ph.random_ellipsoids((16, 16, 16), count=2, rmin=2, rmax=5, dn_max=0.04, seed=5))
f = to_dev(torch, f64, torch.float32)
plan = ls.Plan((16, 16, 16), KB, H)
x = plan.plane_waves(ph.cone_directions(2, 0.8) * KB)
y = torch.empty_like(x)
ls.ls_debug_inject(plan.handle, ls.LS_INJECT_BOUNDS_PROBE, 1)
ls.ls_matvec_batch(plan.handle, f, x, y)
torch.cuda.synchronize()
checked, site = ls.ls_debug_bounds(clear=True)
assert checked and site == 0x601, hex(site)
ls.ls_debug_inject(plan.handle, ls.LS_INJECT_NONE, 0)
ls.ls_matvec_batch(plan.handle, f, x, y)
y1 = torch.empty_like(x[0])
ls.ls_matvec(plan.handle, f, x[1], y1)
torch.cuda.synchronize()
assert rel(y[1].cpu().numpy(), y1.cpu().numpy()) < 1e-6
checked, site = ls.ls_debug_bounds(clear=True)
assert checked and site == 0, hex(site)
plan.close()
print("probe ok", flush=True)
'''


@pytest.mark.gpu
def test_debug_build_checks_pass_on_every_variant_and_report_a_failed_check(tmp_path):
    torch_and_lib()
    import __graft_entry__

    __graft_entry__._build_module().build(debug=True)
    env = dict(os.environ, LS_DEBUG_BOUNDS="1", LS_ROOT=ROOT, LS_AUTOTUNE_CACHE=str(tmp_path / "tune.txt"))
    env["PYTHONPATH"] = ROOT + os.pathsep + os.path.join(ROOT, "tests") + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(CHILD)], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    for name in ("defaults", "variants", "dynamic z", "bead length 144", "z length 128", "z length 192",
                 "z length 384", "non-cubic", "probe"):
        assert f"{name} ok" in r.stdout, r.stdout
