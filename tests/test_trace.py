"""NVTX ranges: every public call, every batched solve and every pass launch opens a named range.

An NVTX injection library (tests/nvtx_record.c, built with the host compiler) records the pushes
and pops of a child process that calls the library."""
import os
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _recorder(tmp_path):
    lib = tmp_path / "libnvtx_record.so"
    r = subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", os.path.join(CUDA_HOME, "include"),
                        os.path.join(HERE, "nvtx_record.c"), "-o", str(lib)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"cannot build the NVTX recorder: {r.stderr.strip()[:200]}")
    return lib


def _run(tmp_path, code):
    lib = _recorder(tmp_path)
    out = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(lib), NVTX_RECORD_FILE=str(out))
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = out.read_text().splitlines() if out.exists() else []
    return lines


def _balanced(lines):
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        assert depth >= 0, "pop without push"
    return depth == 0


def _pushed(lines):
    return [ln[5:] for ln in lines if ln.startswith("push ")]


def test_public_calls_open_ranges_without_a_gpu(tmp_path):
    # argument errors return before any CUDA call, after the call's range has been opened
    lines = _run(tmp_path, """
        import ctypes as C
        from paper_1910_13844_gb300 import _abi
        lib = _abi.load()
        assert lib.ls_forward(None, None, 1, None, None, None, None, None) != 0
        assert lib.ls_gradient(None, None, 1, None, None, None, None, None, None, None, None) != 0
        assert lib.ls_matvec(None, None, None, None, 0, None) != 0
    """)
    names = _pushed(lines)
    assert {"ls_forward", "ls_gradient", "ls_matvec"} <= set(names), names
    assert _balanced(lines)


@pytest.mark.gpu
def test_solve_and_pass_ranges_nest_inside_the_call(tmp_path):
    lines = _run(tmp_path, """
        import numpy as np, torch
        import paper_1910_13844_gb300 as ls
        plan = ls.Plan((16, 16, 16), 8.0, 0.1, use_graphs=0)
        f = torch.full((16, 16, 16), 0.5, device="cuda")
        k = np.array([[0.0, 0.0, 8.0], [1.0, 0.0, 7.9]])
        u, far, code, _ = plan.forward(f, plan.plane_waves(k))
        torch.cuda.synchronize()
        assert code == ls.LS_OK
        plan.close()
    """)
    assert _balanced(lines)
    names = _pushed(lines)
    assert "ls_forward" in names and "solve" in names
    # inside ls_forward: the solve, and in it the five passes, the update and the scalar steps
    i0 = names.index("ls_forward")
    inner = set(names[i0 + 1:])
    assert {"solve", "FX", "FY", "Z", "IY", "IX", "update", "scalar", "far"} <= inner, sorted(inner)
