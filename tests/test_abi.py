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


def test_every_entry_point_rejects_bad_arguments_without_a_gpu(lib):
    # each call below fails its argument check, which comes before any CUDA call
    import ctypes as C

    from paper_1910_13844_gb300 import _abi

    L = _abi.load()
    E = _abi.LS_EINVAL
    g = _abi.ls_grid(16, 16, 16)
    bad_grid = _abi.ls_grid(0, 16, 16)
    one = (C.c_void_p * 1)(None)
    k = (C.c_double * 3)(0.0, 0.0, 15.7)
    assert L.ls_green_spectrum(None, 4, None, None) == E
    assert L.ls_scattering_potential(None, 10, 1.333, 15.7, None, None) == E
    assert L.ls_scattering_potential(None, 0, 1.333, 15.7, None, None) == _abi.LS_OK   # nothing to do
    assert L.ls_plane_waves(None, 1, k, one, None) == E
    assert L.ls_apply_green(None, None, None, 0, None) == E
    assert L.ls_matvec(None, None, None, None, 0, None) == E
    assert L.ls_matvec_noalloc(None, None, None, None, 0, None) == E
    assert L.ls_matvec_batch(None, None, 1, one, one, 0, None) == E
    assert L.ls_forward(None, None, 1, one, one, one, None, None) == E
    assert L.ls_forward_warm(None, None, 1, one, one, one, one, None, None) == E
    assert L.ls_farfield(None, None, 1, one, one, None) == E
    assert L.ls_farfield_adjoint(None, 1, one, one, None) == E
    assert L.ls_residual(0, 16, one, one, one, None, None) == E
    assert L.ls_residual(1, 16, one, one, one, None, None) == E   # null view pointers
    assert L.ls_gradient(None, None, 1, one, one, one, None, None, None, None) == E
    assert L.ls_prox_tv(None, None, None, 0.1, 10, None, None) == E
    assert L.ls_prox_tv(C.byref(bad_grid), None, None, 0.1, 10, None, None) == E
    assert L.ls_prox_hs(C.byref(g), None, None, 0.1, 10, None, None) == E
    assert L.ls_set_pupil(None, 1.0, 0.0) == E
    assert L.ls_apply_pupil(None, 1, one, one, 0, None) == E
    assert L.ls_incident_field(None, 1, one, k, one, None) == E
    assert L.ls_profile(None, 1, None) == E
    t = _abi.ls_tune()
    assert L.ls_autotune(None, 1, None, C.byref(t), None) == E
    srv = C.c_void_p()
    opt = _abi.ls_server_options(k_b=15.7, voxel=0.25)   # k_b h > pi
    assert L.ls_server_create(C.byref(opt), C.byref(srv)) == E
    assert L.ls_server_create(None, C.byref(srv)) == E
    ticket = C.c_uint64()
    assert L.ls_submit(None, None, C.byref(ticket)) == E
    assert L.ls_poll(None, 0, None) == E
    assert L.ls_last_error()   # a message for the last failure


def test_normal_build_reports_no_index_checks_without_a_gpu(lib):
    from paper_1910_13844_gb300 import _abi

    site = ctypes.c_uint(7)
    assert _abi.load().ls_debug_bounds(ctypes.byref(site), 1) == 0
    assert site.value == 0


def test_debug_build_exports_the_same_symbols(repo_root):
    # the index-checking variant is the same library compiled with LS_DEBUG_BOUNDS (no GPU needed to build)
    import __graft_entry__

    path = __graft_entry__._build_module().build(debug=True)
    assert path.endswith("libls_debug.so")
    dbg = ctypes.CDLL(path)
    missing = [n for n in _declared(repo_root) if not hasattr(dbg, n)]
    assert not missing, missing
