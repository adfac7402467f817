"""Shared-memory layout of the TMA-staged z pass (csrc/passes.cuh, ZW<L>), checked on the host for
every length: 16-byte aligned regions, no overlaps, exchange rows inside their pitch, and the
resident CTAs the launch bounds ask for within one SM's shared memory. Needs nvcc but no GPU."""
import os
import shutil
import subprocess

import pytest


def test_z_pass_shared_memory_layout(tmp_path, repo_root):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "zw_layout"
    src = os.path.join(repo_root, "tests", "zw_layout_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(repo_root, "include"),
                        "-I", os.path.join(repo_root, "paper_1910_13844_gb300", "csrc"), src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("OK")
