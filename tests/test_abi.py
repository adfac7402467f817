"""The C-ABI library builds, loads without a GPU and exports every function declared in include/ls.h."""
import ctypes
import os
import re

import pytest


def _declared(repo_root):
    with open(os.path.join(repo_root, "include", "ls.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib(repo_root):
    import __graft_entry__

    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib, repo_root):
    names = _declared(repo_root)
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_functions(repo_root):
    from paper_1910_13844_gb300 import _abi

    assert sorted(_abi.SIGNATURES) == _declared(repo_root)


def test_status_strings_and_defaults_without_gpu(lib):
    from paper_1910_13844_gb300 import _abi

    _abi.load()
    assert _abi.load().ls_status_string(0) == b"LS_OK"
    assert b"NOT_CONVERGED" in _abi.load().ls_status_string(4)
    o = _abi.ls_options()
    _abi.load().ls_default_options(ctypes.byref(o))
    assert o.tol == 1e-6 and o.max_iter == 1000 and o.oversample_p == 4 and o.use_graphs == 1


def test_workspace_estimate_scales_with_views(lib):
    from paper_1910_13844_gb300 import _abi

    g = _abi.ls_grid(128, 128, 128)
    one = _abi.load().ls_workspace_bytes(ctypes.byref(g), 1)
    sixty = _abi.load().ls_workspace_bytes(ctypes.byref(g), 60)
    assert sixty > 50 * (one - (sixty - one) / 59) and sixty < 60 * one


def test_argument_errors_are_reported_without_touching_a_gpu(lib):
    # invalid arguments are rejected before any CUDA call
    from paper_1910_13844_gb300 import _abi

    L = _abi.load()
    g = _abi.ls_grid(20, 20, 20)   # 2n = 40 has no FFT length
    out = ctypes.c_void_p()
    assert L.ls_plan_create(ctypes.byref(g), 2, 15.7, 0.0665, None, ctypes.byref(out)) == _abi.LS_EUNSUPPORTED
    g = _abi.ls_grid(32, 32, 32)
    assert L.ls_plan_create(ctypes.byref(g), 4, 15.7, 0.0665, None, ctypes.byref(out)) == _abi.LS_EINVAL
    assert L.ls_plan_create(ctypes.byref(g), 2, 15.7, 0.25, None, ctypes.byref(out)) == _abi.LS_EINVAL  # k_b h > pi
    assert b"pi" in L.ls_last_error()
    t = _abi.ls_tune()
    assert L.ls_autotune(None, 4, None, ctypes.byref(t), None) == _abi.LS_EINVAL
