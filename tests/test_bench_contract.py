"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON line with the keys the
benchmark contract asks for; run on the small workload, no GPU needed."""
import json
import os
import subprocess
import sys


def test_reference_arm_json_line(repo_root):
    r = subprocess.run([sys.executable, os.path.join(repo_root, "bench.py"), "--impl", "reference", "--workload",
                        "small", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, cwd=repo_root,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("LS forward+adjoint, 32x32x32")


def test_reference_arm_under_two_ranks_runs_on_rank_zero_only(repo_root):
    cmd = [sys.executable, os.path.join(repo_root, "bench.py"), "--impl", "reference", "--workload", "small",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    outs = {}
    for rank in (1, 0):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
        r = subprocess.run(cmd, capture_output=True, text=True, cwd=repo_root, timeout=600, env=env)
        assert r.returncode == 0, r.stderr
        outs[rank] = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert outs[1] == []
    assert len(outs[0]) == 1
    d = json.loads(outs[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["config"]["oracle_processes"] == 1
    assert "rank 0 alone" in d["cpu_baseline"]["sample"]
