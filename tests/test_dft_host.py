"""The register DFTs of the pencil passes (csrc/dft.cuh), compiled as host code, against a direct DFT.

Covers every radix the passes use, with the pruned variants for zero-padded
inputs (unread inputs are NaN, so reading one would show) and cropped outputs.
Needs nvcc but no GPU.
"""
import os
import shutil
import subprocess

import pytest


def test_register_dfts_match_direct_dft(tmp_path, repo_root):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which("nvcc"):
        pytest.skip("nvcc not available")
    exe = tmp_path / "dft_check"
    src = os.path.join(repo_root, "tests", "dft_host_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(repo_root, "include"),
                        "-I", os.path.join(repo_root, "paper_1910_13844_gb300", "csrc"), "-x", "cu", src,
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
