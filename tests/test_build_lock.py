"""Concurrent library builds (one per rank of a multi-process launch) are serialised by a file lock."""
import os
import subprocess
import sys
import time

HOLD = """
import importlib.util, sys, time
spec = importlib.util.spec_from_file_location("b", sys.argv[1]); b = importlib.util.module_from_spec(spec)
spec.loader.exec_module(b)
with b._exclusive(sys.argv[2]):
    print("held", flush=True)
    time.sleep(1.5)
"""

TAKE = """
import importlib.util, sys, time
spec = importlib.util.spec_from_file_location("b", sys.argv[1]); b = importlib.util.module_from_spec(spec)
spec.loader.exec_module(b)
t = time.perf_counter()
with b._exclusive(sys.argv[2]):
    print(time.perf_counter() - t)
"""


def test_a_second_builder_waits_for_the_first(tmp_path, repo_root):
    script = os.path.join(repo_root, "paper_1910_13844_gb300", "build.py")
    lock = str(tmp_path / "lock")
    holder = subprocess.Popen([sys.executable, "-c", HOLD, script, lock], stdout=subprocess.PIPE, text=True)
    try:
        assert holder.stdout.readline().strip() == "held"
        r = subprocess.run([sys.executable, "-c", TAKE, script, lock], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stderr
        waited = float(r.stdout.strip())
        assert waited > 0.5
    finally:
        holder.wait(timeout=60)
    assert holder.returncode == 0
    # once released the lock is taken at once
    t = time.perf_counter()
    r = subprocess.run([sys.executable, "-c", TAKE, script, lock], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and float(r.stdout.strip()) < 0.5
    assert time.perf_counter() - t < 30
