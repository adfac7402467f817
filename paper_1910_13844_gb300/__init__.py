"""GB300 Lippmann-Schwinger forward model and gradient (arXiv 1910.13844).

Thin Python binding of the C ABI in ``include/ls.h``: every function here has
the C name, marshals torch tensors (device memory) and Python lists into
pointers, and calls the CUDA library ``libls.so``.  All arithmetic runs in the
library's kernels; if the library is missing the import fails.

Volumes are torch tensors of shape (nz, ny, nx): complex64 fields, float32
potentials.  Detector arrays are (my, mx) complex64.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import (LS_BREAKDOWN, LS_EAGAIN, LS_ECUDA, LS_EINVAL, LS_ENOMEM, LS_ENOTFOUND, LS_EUNSUPPORTED,
                   LS_INJECT_ALLOC_FAIL, LS_INJECT_BOUNDS_PROBE, LS_INJECT_MAX_ROUNDS, LS_INJECT_NONE, LS_INJECT_Z_STALL,
                   LS_INJECT_ZERO_SHADOW, LS_NOT_CONVERGED, LS_OK, LS_PENDING, LS_REQ_FORWARD, LS_REQ_GRADIENT,
                   LS_TIMEOUT, ls_grid, ls_options, ls_request, ls_result, ls_server_options, ls_stats)

_lib = _abi.load()

__all__ = [
    "LsError", "Plan", "ls_default_options", "ls_plan_create", "ls_plan_destroy", "ls_green_spectrum",
    "ls_scattering_potential", "ls_plane_waves", "ls_apply_green", "ls_matvec", "ls_forward", "ls_farfield",
    "ls_farfield_adjoint", "ls_residual", "ls_gradient", "ls_server_create", "ls_submit", "ls_poll",
    "ls_server_destroy", "ls_status_string", "ls_last_error", "ls_workspace_bytes", "ls_profile", "library_path",
    "ls_matvec_noalloc", "ls_matvec_batch", "Server", "ls_set_pupil", "ls_apply_pupil", "ls_incident_field",
    "ls_forward_warm", "ls_prox_tv", "ls_prox_hs", "ls_autotune", "ls_inner_products", "ls_debug_inject",
    "ls_fp32_peak", "ls_debug_bounds",
]

_SOFT = (LS_OK, LS_NOT_CONVERGED, LS_BREAKDOWN, LS_TIMEOUT, LS_PENDING)


class LsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.ls_status_string(code).decode()
        detail = _lib.ls_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def _check(code: int, where: str) -> int:
    if code not in _SOFT:
        raise LsError(code, where)
    return code


def library_path() -> str:
    return _abi.LIB_PATH


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("tensor must be on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    raise TypeError(f"expected a CUDA tensor or an integer device pointer, got {type(t)}")


def _views(ts):
    """Host array of device pointers for a list of tensors / a [Q, ...] tensor, or None."""
    if ts is None:
        return None, 0
    if isinstance(ts, torch.Tensor):
        ts = list(ts.unbind(0)) if ts.dim() >= 2 and ts.is_contiguous() else [ts]
    ptrs = [_ptr(t) for t in ts]
    arr = (C.c_void_p * len(ptrs))(*ptrs)
    return arr, len(ptrs)


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def ls_status_string(code: int) -> str:
    return _lib.ls_status_string(int(code)).decode()


def ls_last_error() -> str:
    return _lib.ls_last_error().decode()


def ls_default_options(**overrides) -> ls_options:
    o = ls_options()
    _lib.ls_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def ls_workspace_bytes(grid, n_views: int) -> int:
    g = ls_grid(*grid)
    return int(_lib.ls_workspace_bytes(C.byref(g), int(n_views)))


def ls_plan_create(grid, padding: int, k_b: float, voxel: float, opt: ls_options | None = None) -> int:
    """grid = (nx, ny, nz).  Returns the plan handle (int)."""
    g = ls_grid(*[int(v) for v in grid])
    out = C.c_void_p()
    _check(_lib.ls_plan_create(C.byref(g), int(padding), float(k_b), float(voxel),
                               C.byref(opt) if opt is not None else None, C.byref(out)), "ls_plan_create")
    return out.value


def ls_plan_destroy(plan: int) -> None:
    _lib.ls_plan_destroy(plan)


def ls_green_spectrum(plan: int, oversample_p: int, out=None, stream=None) -> int:
    return _check(_lib.ls_green_spectrum(plan, int(oversample_p), _ptr(out), _stream(stream)), "ls_green_spectrum")


def ls_scattering_potential(dn, eta_b: float, k_b: float, f, stream=None) -> int:
    return _check(_lib.ls_scattering_potential(_ptr(dn), dn.numel(), float(eta_b), float(k_b), _ptr(f),
                                               _stream(stream)), "ls_scattering_potential")


def ls_plane_waves(plan: int, kvec, u_in, stream=None) -> int:
    k = np.ascontiguousarray(np.asarray(kvec, dtype=np.float64).reshape(-1, 3))
    arr, n = _views(u_in)
    if n != k.shape[0]:
        raise ValueError("one wave vector per view")
    return _check(_lib.ls_plane_waves(plan, n, k.ctypes.data_as(C.POINTER(C.c_double)), arr, _stream(stream)),
                  "ls_plane_waves")


def ls_apply_green(plan: int, v, out, adjoint: bool = False, stream=None) -> int:
    return _check(_lib.ls_apply_green(plan, _ptr(v), _ptr(out), int(bool(adjoint)), _stream(stream)),
                  "ls_apply_green")


def ls_matvec(plan: int, f, x, y, adjoint: bool = False, stream=None) -> int:
    return _check(_lib.ls_matvec(plan, _ptr(f), _ptr(x), _ptr(y), int(bool(adjoint)), _stream(stream)), "ls_matvec")


def ls_set_pupil(plan: int, k_cut: float, distance: float = 0.0) -> int:
    """Pupil of cut-off k_cut (1/um) and refocus over `distance` um applied to every far field (P of eq. lipp2)."""
    return _check(_lib.ls_set_pupil(plan, float(k_cut), float(distance)), "ls_set_pupil")


def ls_apply_pupil(plan: int, x, y, adjoint: bool = False, stream=None) -> int:
    ax, n = _views(x)
    ay, _ = _views(y)
    return _check(_lib.ls_apply_pupil(plan, n, ax, ay, int(bool(adjoint)), _stream(stream)), "ls_apply_pupil")


def ls_incident_field(plan: int, y_in, u_in, k_in=None, stream=None) -> int:
    """u_in (Q, nz, ny, nx) from detector fields y_in (Q, ny, nx); k_in (Q, 2) enables tilt transfer."""
    ay, n = _views(y_in)
    au, _ = _views(u_in)
    karr, kptr = None, None
    if k_in is not None:
        karr = np.ascontiguousarray(np.asarray(k_in, dtype=np.float64).reshape(-1, 2))
        if karr.shape[0] != n:
            raise ValueError("one lateral wave vector per view")
        kptr = karr.ctypes.data_as(C.POINTER(C.c_double))
    return _check(_lib.ls_incident_field(plan, n, ay, kptr, au, _stream(stream)), "ls_incident_field")


def ls_matvec_batch(plan: int, f, x, y, adjoint: bool = False, stream=None) -> int:
    """y[q] = x[q] - G (f x[q]) for a list / [Q, ...] tensor of vectors, one batched launch per pass."""
    ax, n = _views(x)
    ay, m = _views(y)
    if n != m:
        raise ValueError("x and y need the same number of views")
    return _check(_lib.ls_matvec_batch(plan, _ptr(f), n, ax, ay, int(bool(adjoint)), _stream(stream)),
                  "ls_matvec_batch")


def ls_matvec_noalloc(plan: int, f, x, y, adjoint: bool = False, stream=None) -> int:
    """ls_matvec without any device allocation (static scratch inside the library, grids up to 1398101 voxels)."""
    return _check(_lib.ls_matvec_noalloc(plan, _ptr(f), _ptr(x), _ptr(y), int(bool(adjoint)), _stream(stream)),
                  "ls_matvec_noalloc")


def ls_forward(plan: int, f, u_in, u_out=None, far=None, stream=None, n_views=None):
    """Returns (status, [stats dict per view]).  u_in None: the plan's built-in plane waves for n_views views."""
    a_in, n = _views(u_in)
    if u_in is None:
        if not n_views:
            raise ValueError("n_views is needed when u_in is None")
        n = int(n_views)
    a_out, _ = _views(u_out)
    a_far, _ = _views(far)
    st = (ls_stats * n)()
    code = _check(_lib.ls_forward(plan, _ptr(f), n, a_in, a_out, a_far, st, _stream(stream)), "ls_forward")
    return code, [s.as_dict() for s in st]


def ls_forward_warm(plan: int, f, u_in, x0, u_out=None, far=None, stream=None):
    """ls_forward starting BiCGStab from x0 (Q, nz, ny, nx); x0 may be u_out.  Returns (status, stats)."""
    a_in, n = _views(u_in)
    a_x0, n0 = _views(x0)
    if n0 != n:
        raise ValueError("one initial guess per view")
    a_out, _ = _views(u_out)
    a_far, _ = _views(far)
    st = (ls_stats * n)()
    code = _check(_lib.ls_forward_warm(plan, _ptr(f), n, a_in, a_x0, a_out, a_far, st, _stream(stream)),
                  "ls_forward_warm")
    return code, [s.as_dict() for s in st]


def ls_prox_tv(z, x, lam: float, iters: int = 20, work=None, stream=None) -> int:
    """x = prox of lam TV + i_{>=0} at z (float32 CUDA tensors (nz, ny, nx)) by `iters` FGP iterations."""
    if z.dim() != 3 or z.shape != x.shape:
        raise ValueError("z and x must be (nz, ny, nx) tensors of the same shape")
    nz, ny, nx = z.shape
    g = ls_grid(nx, ny, nz)
    return _check(_lib.ls_prox_tv(C.byref(g), _ptr(z), _ptr(x), float(lam), int(iters),
                                  _ptr(work) if work is not None else None, _stream(stream)), "ls_prox_tv")


def ls_prox_hs(z, x, lam: float, iters: int = 20, work=None, stream=None) -> int:
    """x = prox of lam * (Hessian Schatten-1 norm) + i_{>=0} at z (float32 CUDA (nz, ny, nx)), FGP."""
    if z.dim() != 3 or z.shape != x.shape:
        raise ValueError("z and x must be (nz, ny, nx) tensors of the same shape")
    nz, ny, nx = z.shape
    g = ls_grid(nx, ny, nz)
    return _check(_lib.ls_prox_hs(C.byref(g), _ptr(z), _ptr(x), float(lam), int(iters),
                                  _ptr(work) if work is not None else None, _stream(stream)), "ls_prox_hs")


def ls_autotune(plan: int, n_views: int, f, stream=None) -> dict:
    """Time the plan's launch variants for batches of n_views views of f and keep the fastest.

    Returns the chosen variants and timings (ls_tune as a dict).  With LS_AUTOTUNE_CACHE set to a
    file name, results are read from / appended to that file."""
    t = _abi.ls_tune()
    _check(_lib.ls_autotune(plan, int(n_views), _ptr(f), C.byref(t), _stream(stream)), "ls_autotune")
    return t.as_dict()


def ls_farfield(plan: int, f, u, far, stream=None) -> int:
    a_u, n = _views(u)
    a_far, _ = _views(far)
    return _check(_lib.ls_farfield(plan, _ptr(f), n, a_u, a_far, _stream(stream)), "ls_farfield")


def ls_farfield_adjoint(plan: int, r, out, stream=None) -> int:
    a_r, n = _views(r)
    a_o, _ = _views(out)
    return _check(_lib.ls_farfield_adjoint(plan, n, a_r, a_o, _stream(stream)), "ls_farfield_adjoint")


def ls_residual(pred, meas, res, stream=None):
    """res = pred - meas per view; returns per-view ||res||^2 (float64 numpy array)."""
    a_p, n = _views(pred)
    a_m, _ = _views(meas)
    a_r, _ = _views(res)
    count = (pred[0] if isinstance(pred, (list, tuple)) else pred[0]).numel()
    loss = (C.c_double * n)()
    _check(_lib.ls_residual(n, count, a_p, a_m, a_r, loss, _stream(stream)), "ls_residual")
    return np.array(loss[:], dtype=np.float64)


def ls_inner_products(a, b, stream=None):
    """<a[q], b[q]> = sum conj(a[q]) b[q] per view (complex128 numpy array), the solver's inner product."""
    a_a, n = _views(a)
    a_b, m = _views(b)
    if n != m:
        raise ValueError("a and b need the same number of views")
    count = (a[0] if isinstance(a, (list, tuple)) else a[0]).numel()
    out = (C.c_double * (2 * n))()
    _check(_lib.ls_inner_products(n, count, a_a, a_b, out, _stream(stream)), "ls_inner_products")
    v = np.array(out[:], dtype=np.float64)
    return v[0::2] + 1j * v[1::2]


def ls_fp32_peak(stream=None) -> dict:
    """Measured FP32 lane operations per second of the current device: FFMA, FMUL, packed add.f32x2."""
    out = (C.c_double * 3)()
    _check(_lib.ls_fp32_peak(out, _stream(stream)), "ls_fp32_peak")
    return {"ffma": out[0], "fmul": out[1], "fadd2": out[2]}


def ls_debug_bounds(clear: bool = False):
    """(checked, site): checked is True in the index-checking build (LS_DEBUG_BOUNDS=1); site is the
    first failed check's code (0: none)."""
    site = C.c_uint(0)
    rc = _lib.ls_debug_bounds(C.byref(site), int(bool(clear)))
    if rc < 0 or rc > 1:
        _check(rc, "ls_debug_bounds")
    return bool(rc), int(site.value)


def ls_debug_inject(plan, kind: int, value: int = 0) -> int:
    """Test-only failure injection (LS_INJECT_* kinds of include/ls.h); plan may be None for ALLOC_FAIL."""
    return _check(_lib.ls_debug_inject(plan, int(kind), int(value)), "ls_debug_inject")


def ls_gradient(plan: int, f, residuals, grad, u_in=None, u_fwd=None, view_weights=None, stream=None):
    """Returns (status, [stats dict per view]) and writes grad."""
    a_r, n = _views(residuals)
    a_in, _ = _views(u_in)
    a_fw, _ = _views(u_fwd)
    w = None
    if view_weights is not None:
        w = (C.c_double * n)(*[float(x) for x in view_weights])
    st = (ls_stats * n)()
    code = _check(_lib.ls_gradient(plan, _ptr(f), n, a_in, a_fw, a_r, w, _ptr(grad), st, _stream(stream)),
                  "ls_gradient")
    return code, [s.as_dict() for s in st]


def ls_profile(plan: int, enable: bool):
    """Turn per-launch event timing on/off.

    Returns {kind: (ms, launches, slot_passes, active_slot_passes)} accumulated so far."""
    t = _abi.ls_kernel_times()
    _check(_lib.ls_profile(plan, int(bool(enable)), C.byref(t)), "ls_profile")
    return {name: (t.ms[i], t.launches[i], t.slot_passes[i], t.active_slot_passes[i])
            for i, name in enumerate(_abi.LS_K_NAMES)}


def ls_server_create(opt: ls_server_options) -> int:
    out = C.c_void_p()
    _check(_lib.ls_server_create(C.byref(opt), C.byref(out)), "ls_server_create")
    return out.value


def ls_submit(server: int, req: ls_request) -> tuple[int, int]:
    t = C.c_uint64()
    code = _lib.ls_submit(server, C.byref(req), C.byref(t))
    if code not in (LS_OK, LS_EAGAIN):
        raise LsError(code, "ls_submit")
    return code, t.value


def ls_poll(server: int, ticket: int):
    r = ls_result()
    code = _lib.ls_poll(server, C.c_uint64(ticket), C.byref(r))
    if code == LS_ENOTFOUND:
        raise LsError(code, "ls_poll")
    return code, {"status": r.status, "iterations_max": r.iterations_max, "ms": r.submit_to_done_ms}


def ls_server_destroy(server: int) -> None:
    _lib.ls_server_destroy(server)


class Plan:
    """Owning wrapper of an ls_plan for one grid (shape given as (nz, ny, nx))."""

    def __init__(self, shape, k_b: float, voxel: float, **options):
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.k_b = float(k_b)
        self.voxel = float(voxel)
        self.options = ls_default_options(**options)
        self.handle = ls_plan_create((nx, ny, nz), 2, k_b, voxel, self.options)
        self.det = (self.options.det_my or ny, self.options.det_mx or nx)

    def close(self):
        if getattr(self, "handle", None):
            ls_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience allocations
    def field(self, n=None, device="cuda"):
        s = self.shape if n is None else (n,) + self.shape
        return torch.empty(s, dtype=torch.complex64, device=device)

    def detector(self, n=None, device="cuda"):
        s = self.det if n is None else (n,) + self.det
        return torch.empty(s, dtype=torch.complex64, device=device)

    def plane_waves(self, kvec, stream=None):
        k = np.asarray(kvec, dtype=np.float64).reshape(-1, 3)
        u = self.field(k.shape[0])
        ls_plane_waves(self.handle, k, u, stream)
        return u

    def forward(self, f, u_in, want_fields=True, want_far=True, stream=None, n_views=None):
        """u_in None: the built-in plane waves (options cone_sin_theta) for n_views views."""
        q = u_in.shape[0] if u_in is not None else int(n_views)
        u = self.field(q) if want_fields else None
        far = self.detector(q) if want_far else None
        code, stats = ls_forward(self.handle, f, u_in, u, far, stream, n_views=q)
        return u, far, code, stats

    def autotune(self, n_views: int, f, stream=None) -> dict:
        return ls_autotune(self.handle, n_views, f, stream)

    def gradient(self, f, residuals, u_fwd=None, u_in=None, weights=None, stream=None):
        g = torch.empty(self.shape, dtype=torch.float32, device=f.device)
        code, stats = ls_gradient(self.handle, f, residuals, g, u_in=u_in, u_fwd=u_fwd, view_weights=weights,
                                  stream=stream)
        return g, code, stats


class Server:
    """Owning wrapper of an ls_server (continuous batching of forward and gradient requests).

    Tensors passed to ``submit_*`` must stay alive until ``poll`` reports the
    request finished; this wrapper keeps references to them until then.
    """

    def __init__(self, k_b: float, voxel: float, tol: float = 1e-6, max_iter: int = 1000,
                 hbm_budget_bytes: int = 0, max_views_per_grid: int = 0, iters_per_round: int = 0):
        opt = ls_server_options(hbm_budget_bytes=hbm_budget_bytes, max_views_per_grid=max_views_per_grid,
                                tol=tol, max_iter=max_iter, k_b=k_b, voxel=voxel, iters_per_round=iters_per_round)
        self.handle = ls_server_create(opt)
        self._keep = {}

    def _submit(self, kind, f, kvec, meas=None, u_out=None, far=None, grad=None):
        nz, ny, nx = f.shape
        k = np.ascontiguousarray(np.asarray(kvec, dtype=np.float64).reshape(-1, 3))
        loss = C.c_double(float("nan"))
        req = ls_request(kind=kind, grid=ls_grid(nx, ny, nz), n_views=k.shape[0], f=_ptr(f),
                         kvec=k.ctypes.data_as(C.POINTER(C.c_double)), meas=_ptr(meas), u_out=_ptr(u_out),
                         far=_ptr(far), grad=_ptr(grad), loss=C.pointer(loss))
        code, ticket = ls_submit(self.handle, req)
        if code != LS_OK:
            raise LsError(code, "ls_submit")
        self._keep[ticket] = (f, k, meas, u_out, far, grad, loss)
        return ticket

    def submit_forward(self, f, kvec, u_out=None, far=None) -> int:
        return self._submit(LS_REQ_FORWARD, f, kvec, u_out=u_out, far=far)

    def submit_gradient(self, f, kvec, meas, grad, u_out=None) -> int:
        return self._submit(LS_REQ_GRADIENT, f, kvec, meas=meas, grad=grad, u_out=u_out)

    def poll(self, ticket: int):
        """(status, info) with status LS_PENDING while running; info has 'ms', 'iterations_max', 'loss'."""
        code, info = ls_poll(self.handle, ticket)
        if code != LS_PENDING:
            keep = self._keep.pop(ticket, None)
            info["loss"] = keep[6].value if keep is not None else float("nan")
        return code, info

    def wait(self, ticket: int, timeout_s: float = 600.0):
        import time as _t
        t0 = _t.time()
        while True:
            code, info = self.poll(ticket)
            if code != LS_PENDING:
                return code, info
            if _t.time() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} still pending after {timeout_s} s")
            _t.sleep(0.0005)

    def close(self):
        if getattr(self, "handle", None):
            ls_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
