"""bench.py's host-side arithmetic: the FP32-pipe roofline, the source-keyed ncu records and the
seeded serving mix (no GPU needed)."""
import importlib.util
import json
import os
import sys

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bench(repo_root):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(repo_root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_alu_roofline_floor_and_fraction(bench):
    # equal rates for every instruction kind: the peak is that rate; a packed FADD2 is 64 lane operations
    ops = {"fadd2": 2.0e6, "ffma": 1.0e6, "fmul": 0.5e6}
    rate = {"fadd2": 40e12, "ffma": 40e12, "fmul": 40e12}
    lane_ops = 64 * 2.0e6 + 32 * 1.0e6 + 32 * 0.5e6
    r = bench.alu_roofline(ops, launch_ms=2.0, views_per_launch=10, fp32_peak=rate, sm_count=152)
    assert r["ops_per_view"] == int(lane_ops)
    assert r["peak"] == pytest.approx(40.0, rel=1e-9)
    assert r["achieved"] == pytest.approx(lane_ops * 10 / 2e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    # a slower FADD2 lowers the peak to the time-weighted harmonic mean of the rates
    rate2 = dict(rate, fadd2=20e12)
    r2 = bench.alu_roofline(ops, 2.0, 10, rate2, 152)
    floor = 64 * 2.0e6 / 20e12 + 32 * 1.0e6 / 40e12 + 32 * 0.5e6 / 40e12
    assert r2["peak"] == pytest.approx(lane_ops / floor / 1e12, rel=1e-3)
    assert bench.alu_roofline(None, 2.0, 10, rate, 152) is None


def test_ncu_records_are_used_only_for_the_sources_they_were_taken_on(bench, tmp_path, monkeypatch):
    for f in bench.Z_SOURCES:
        p = tmp_path / f
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text("source " + f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"z_pass": {"dram_bytes_per_slot": 123.0, "fadd2_per_slot": 1.0, "ffma_per_slot": 2.0,
                      "fmul_per_slot": 3.0, "source_hash": bench.source_hash(bench.Z_SOURCES)}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.traffic_per_slot("z_pass") == 123.0
    assert bench.opcodes_per_slot("z_pass") == {"fadd2": 1.0, "ffma": 2.0, "fmul": 3.0}
    # any change to one of the z pass's sources makes the record stale
    (tmp_path / bench.Z_SOURCES[0]).write_text("changed")
    assert bench.traffic_per_slot("z_pass") is None
    assert bench.opcodes_per_slot("z_pass") is None


def test_serving_mix_is_seeded_and_has_the_configured_shape(bench):
    a = bench.serve_requests(2000, seed=2026)
    b = bench.serve_requests(2000, seed=2026)
    assert a == b
    assert {tuple(r["shape"]) for r in a} == {tuple(s) for s in bench.SERVE_GRIDS}
    views = np.array([r["views"] for r in a])
    assert views.min() >= 8 and views.max() <= 60
    grad = np.mean([r["grad"] for r in a])
    assert abs(grad - 0.3) < 0.04
    assert bench.serve_requests(50, seed=1) != bench.serve_requests(50, seed=2)
