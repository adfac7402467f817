"""ctypes declarations of the C ABI in include/ls.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# LS_DEBUG_BOUNDS=1 in the environment selects the index-checking build (libls_debug.so)
DEBUG_BOUNDS = os.environ.get("LS_DEBUG_BOUNDS", "0") == "1"
LIB_PATH = os.path.join(HERE, "libls_debug.so" if DEBUG_BOUNDS else "libls.so")

LS_OK = 0
LS_EINVAL = 1
LS_ENOMEM = 2
LS_ECUDA = 3
LS_NOT_CONVERGED = 4
LS_BREAKDOWN = 5
LS_TIMEOUT = 6
LS_PENDING = 7
LS_EAGAIN = 8
LS_ENOTFOUND = 9
LS_EUNSUPPORTED = 10

LS_INJECT_NONE = 0
LS_INJECT_ZERO_SHADOW = 1
LS_INJECT_MAX_ROUNDS = 2
LS_INJECT_ALLOC_FAIL = 3
LS_INJECT_Z_STALL = 4
LS_INJECT_BOUNDS_PROBE = 5

LS_REQ_FORWARD = 0
LS_REQ_GRADIENT = 1


class ls_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class ls_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("oversample_p", C.c_int),
                ("det_mx", C.c_int), ("det_my", C.c_int), ("x_gamma", C.c_double),
                ("max_restarts", C.c_int), ("check_every", C.c_int), ("use_graphs", C.c_int),
                ("cone_sin_theta", C.c_double)]


class ls_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int), ("matvecs", C.c_int),
                ("rel_residual", C.c_double), ("true_rel_residual", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ls_server_options(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_views_per_grid", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("k_b", C.c_double), ("voxel", C.c_double), ("iters_per_round", C.c_int)]


class ls_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("grid", ls_grid), ("n_views", C.c_int), ("f", C.c_void_p),
                ("kvec", C.POINTER(C.c_double)), ("meas", C.c_void_p), ("u_out", C.c_void_p),
                ("far", C.c_void_p), ("grad", C.c_void_p), ("loss", C.POINTER(C.c_double))]


LS_K_NAMES = ["fx", "fy", "z", "iy", "ix", "update", "scalar", "far", "other"]


class ls_kernel_times(C.Structure):
    _fields_ = [("ms", C.c_double * 9), ("launches", C.c_longlong * 9), ("slot_passes", C.c_longlong * 9),
                ("active_slot_passes", C.c_longlong * 9)]


class ls_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations_max", C.c_int), ("submit_to_done_ms", C.c_double)]


class ls_tune(C.Structure):
    _fields_ = [("z_tma", C.c_int), ("ix_prefetch", C.c_int), ("fx_views_fastest", C.c_int),
                ("check_every", C.c_int), ("use_graphs", C.c_int), ("matvec_us_per_view", C.c_double),
                ("solve_ms", C.c_double), ("from_cache", C.c_int), ("z_split", C.c_int), ("strided_wide", C.c_int),
                ("views_per_launch", C.c_int), ("z_persist", C.c_int), ("fx_bulk", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)

# name -> (restype, argtypes); every function declared in include/ls.h
SIGNATURES = {
    "ls_default_options": (None, [C.POINTER(ls_options)]),
    "ls_plan_create": (C.c_int, [C.POINTER(ls_grid), C.c_int, C.c_double, C.c_double, C.POINTER(ls_options), _PP]),
    "ls_plan_destroy": (None, [_P]),
    "ls_green_spectrum": (C.c_int, [_P, C.c_int, _P, _P]),
    "ls_scattering_potential": (C.c_int, [_P, C.c_size_t, C.c_double, C.c_double, _P, _P]),
    "ls_plane_waves": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), _PP, _P]),
    "ls_apply_green": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "ls_matvec": (C.c_int, [_P, _P, _P, _P, C.c_int, _P]),
    "ls_forward": (C.c_int, [_P, _P, C.c_int, _PP, _PP, _PP, C.POINTER(ls_stats), _P]),
    "ls_forward_warm": (C.c_int, [_P, _P, C.c_int, _PP, _PP, _PP, _PP, C.POINTER(ls_stats), _P]),
    "ls_prox_tv": (C.c_int, [C.POINTER(ls_grid), _P, _P, C.c_double, C.c_int, _P, _P]),
    "ls_prox_hs": (C.c_int, [C.POINTER(ls_grid), _P, _P, C.c_double, C.c_int, _P, _P]),
    "ls_farfield": (C.c_int, [_P, _P, C.c_int, _PP, _PP, _P]),
    "ls_farfield_adjoint": (C.c_int, [_P, C.c_int, _PP, _PP, _P]),
    "ls_residual": (C.c_int, [C.c_int, C.c_size_t, _PP, _PP, _PP, C.POINTER(C.c_double), _P]),
    "ls_gradient": (C.c_int, [_P, _P, C.c_int, _PP, _PP, _PP, C.POINTER(C.c_double), _P,
                              C.POINTER(ls_stats), _P]),
    "ls_server_create": (C.c_int, [C.POINTER(ls_server_options), _PP]),
    "ls_submit": (C.c_int, [_P, C.POINTER(ls_request), C.POINTER(C.c_uint64)]),
    "ls_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(ls_result)]),
    "ls_server_destroy": (None, [_P]),
    "ls_status_string": (C.c_char_p, [C.c_int]),
    "ls_last_error": (C.c_char_p, []),
    "ls_workspace_bytes": (C.c_size_t, [C.POINTER(ls_grid), C.c_int]),
    "ls_profile": (C.c_int, [_P, C.c_int, C.POINTER(ls_kernel_times)]),
    "ls_matvec_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int, _P]),
    "ls_matvec_batch": (C.c_int, [_P, _P, C.c_int, _PP, _PP, C.c_int, _P]),
    "ls_set_pupil": (C.c_int, [_P, C.c_double, C.c_double]),
    "ls_apply_pupil": (C.c_int, [_P, C.c_int, _PP, _PP, C.c_int, _P]),
    "ls_incident_field": (C.c_int, [_P, C.c_int, _PP, C.POINTER(C.c_double), _PP, _P]),
    "ls_autotune": (C.c_int, [_P, C.c_int, _P, C.POINTER(ls_tune), _P]),
    "ls_inner_products": (C.c_int, [C.c_int, C.c_size_t, _PP, _PP, C.POINTER(C.c_double), _P]),
    "ls_debug_inject": (C.c_int, [_P, C.c_int, C.c_longlong]),
    "ls_fp32_peak": (C.c_int, [C.POINTER(C.c_double), _P]),
    "ls_debug_bounds": (C.c_int, [C.POINTER(C.c_uint), C.c_int]),
}

_lib = None


def load() -> C.CDLL:
    """Load ``libls.so`` (``libls_debug.so`` with LS_DEBUG_BOUNDS=1); raises ImportError when the CUDA
    library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run paper_1910_13844_gb300.build.build("
                          f"{'debug=True' if DEBUG_BOUNDS else ''}) (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
