"""Discrete LS forward model, far field and data-fidelity gradient (oracle).

eq. lipp1:  u = (I - G diag(f))^{-1} u_in
eq. lipp2:  y_sc = P G~ diag(f) u           (P = I here)
eq. prob:   loss = sum_q ||H_q(f) - y_q||^2 / (2 ||y_q||^2)
Alg. 1:     d = sum_q Re(J_q^H (H_q(f) - y_q)) / ||y_q||^2

Test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla

from . import kernel as K
from .green import green, wavenumber

_WORKERS = -1


@dataclass
class Setup:
    """Grid and optics of one problem.  ``shape`` is (nz, ny, nx); lengths in micrometres."""

    shape: tuple
    h: float
    kb: float
    p: int = 4
    m: tuple | None = None        # detector (my, mx); default (ny, nx)
    x_gamma: float | None = None  # detector plane z position; default 3 L_z / 4

    @property
    def det(self):
        return self.m if self.m is not None else (self.shape[1], self.shape[2])

    @property
    def zgamma(self):
        return self.x_gamma if self.x_gamma is not None else 0.75 * self.shape[0] * self.h


def setup_from_optics(shape, lam_um: float, eta_b: float, h_um: float, p: int = 4, **kw) -> Setup:
    return Setup(tuple(shape), h_um, wavenumber(lam_um, eta_b), p, **kw)


def coords(shape, h):
    """Physical voxel centres (z, y, x), centred index set (Theorem 1)."""
    nz, ny, nx = shape
    c = lambda n: (np.arange(n) - n // 2 + 1) * h
    return c(nz)[:, None, None], c(ny)[None, :, None], c(nx)[None, None, :]


def plane_wave(shape, h, kvec) -> np.ndarray:
    """u_in(x) = exp(i k . x) at the voxel centres; kvec = (kx, ky, kz) (Fig. 1)."""
    z, y, x = coords(shape, h)
    return np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))


class Operator:
    """G and G~ for one Setup.  G uses the reduced-padding spectrum (Prop. 1); G~ is eq. Gtild-1."""

    def __init__(self, st: Setup, kernel_method: str = "fft"):
        self.st = st
        self.Kern = K.build_green(st.shape, st.h, st.kb, st.p, kernel_method)
        self.Ghat = K.green_spectrum(self.Kern)

    # -- volume operator ---------------------------------------------------
    def G(self, v, adjoint=False):
        return K.apply_G_fft(self.Ghat, v, adjoint)

    def A(self, x, f, adjoint=False):
        """x - G (f x)  (forward, eq. lipp1)  or  x - G^H (f x)  (adjoint system of Alg. 1 line 6)."""
        return x - self.G(f * x, adjoint)

    # -- detector operator -------------------------------------------------
    def detector_points(self):
        my, mx = self.st.det
        h = self.st.h
        ya = (np.arange(my) - my // 2 + 1) * h
        xa = (np.arange(mx) - mx // 2 + 1) * h
        return ya, xa, self.st.zgamma

    def farfield_direct(self, v):
        """y[j] = sum_{z in Omega} h^3 g(x_j - z) v(z), v = f u (midpoint rule of eq. Gtild-1)."""
        st = self.st
        z, y, x = coords(st.shape, st.h)
        ya, xa, zg = self.detector_points()
        out = np.zeros((len(ya), len(xa)), dtype=np.complex128)
        dz2 = (zg - z) ** 2
        for a, yy in enumerate(ya):
            dy2 = (yy - y) ** 2
            for b, xx in enumerate(xa):
                r = np.sqrt(dz2 + dy2 + (xx - x) ** 2)
                out[a, b] = np.sum(green(r, st.kb) * v) * st.h ** 3
        return out

    def farfield_pixels(self, v, pixels):
        """Direct-sum far field at selected detector pixels [(a, b), ...]."""
        st = self.st
        z, y, x = coords(st.shape, st.h)
        ya, xa, zg = self.detector_points()
        out = []
        for a, b in pixels:
            r = np.sqrt((zg - z) ** 2 + (ya[a] - y) ** 2 + (xa[b] - x) ** 2)
            out.append(np.sum(green(r, st.kb) * v) * st.h ** 3)
        return np.array(out)

    def farfield_matrix(self):
        """Explicit M x N matrix of G~ (tiny grids)."""
        st = self.st
        z, y, x = coords(st.shape, st.h)
        ya, xa, zg = self.detector_points()
        Z, Y, X = np.broadcast_arrays(z, y, x)
        Z, Y, X = Z.ravel(), Y.ravel(), X.ravel()
        YA, XA = np.meshgrid(ya, xa, indexing="ij")
        r = np.sqrt((zg - Z[None, :]) ** 2 + (YA.ravel()[:, None] - Y[None, :]) ** 2 + (XA.ravel()[:, None] - X[None, :]) ** 2)
        return green(r, st.kb) * st.h ** 3

    def _slice_kernels(self):
        """Per-slice 2-D kernels h^3 g(h dx, h dy, x_Gamma - z_s), dx, dy in [-(n-1), n-1], on the 2n grid."""
        st = self.st
        nz, ny, nx = st.shape
        zc = (np.arange(nz) - nz // 2 + 1) * st.h
        dy = K.centred(2 * ny).astype(np.float64) * st.h
        dx = K.centred(2 * nx).astype(np.float64) * st.h
        ker = np.empty((nz, 2 * ny, 2 * nx), dtype=np.complex128)
        for s in range(nz):
            r = np.sqrt((st.zgamma - zc[s]) ** 2 + dy[:, None] ** 2 + dx[None, :] ** 2)
            ker[s] = green(r, st.kb) * st.h ** 3
        ker[:, ny, :] = 0.0
        ker[:, :, nx] = 0.0
        return ker

    def farfield_fft(self, v):
        """Same far field as ``farfield_direct``, as a sum over slices of 2-D linear convolutions (Sec. 3.2)."""
        st = self.st
        nz, ny, nx = st.shape
        my, mx = st.det
        oy, ox = (ny - my) // 2, (nx - mx) // 2
        ker = sfft.fft2(self._slice_kernels(), workers=_WORKERS)
        vp = np.zeros((nz, 2 * ny, 2 * nx), dtype=np.complex128)
        vp[:, :ny, :nx] = v
        acc = np.sum(ker * sfft.fft2(vp, workers=_WORKERS), axis=0)
        full = sfft.ifft2(acc, workers=_WORKERS)
        return full[oy:oy + my, ox:ox + mx]

    def farfield_adjoint_fft(self, r):
        """G~^H r: per-slice 2-D correlation with the conjugate kernels."""
        st = self.st
        nz, ny, nx = st.shape
        my, mx = st.det
        oy, ox = (ny - my) // 2, (nx - mx) // 2
        ker = sfft.fft2(self._slice_kernels(), workers=_WORKERS)
        rp = np.zeros((2 * ny, 2 * nx), dtype=np.complex128)
        rp[oy:oy + my, ox:ox + mx] = r
        out = sfft.ifft2(np.conj(ker) * sfft.fft2(rp, workers=_WORKERS)[None], workers=_WORKERS)
        return out[:, :ny, :nx]


# ---------------------------------------------------------------------------
# Solvers for eq. lipp1
# ---------------------------------------------------------------------------

def bicgstab(apply_A, b, x0=None, tol=1e-12, maxiter=1000):
    """Textbook BiCGStab (van der Vorst 1992) in complex128, <a, b> = sum conj(a) b.

    Starts from x0 (default b), stops when ||b - A x|| (recursive) <= tol ||b||.
    Returns (x, iterations, recursive relative residual).
    """
    x = np.array(b if x0 is None else x0, dtype=np.complex128, copy=True)
    r = b - apply_A(x)
    rh = r.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(x), 0, 0.0
    rn = np.linalg.norm(r)
    if rn <= tol * bn:
        return x, 0, rn / bn
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(x)
    p = np.zeros_like(x)
    it = 0
    for it in range(1, maxiter + 1):
        rho_new = np.vdot(rh, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_A(p)
        alpha = rho_new / np.vdot(rh, v)
        s = r - alpha * v
        t = apply_A(s)
        tt = np.vdot(t, t)
        omega = np.vdot(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        rn = np.linalg.norm(r)
        if rn <= tol * bn:
            break
    return x, it, rn / bn


def solve_lu(op: Operator, f, b, adjoint=False):
    """Direct solve of (I - G diag f) u = b (or the adjoint system) with a dense LU (tiny grids)."""
    shape = b.shape
    Gd = K.dense_G(op.Kern, shape)
    if adjoint:
        Gd = np.conj(Gd)
    A = np.eye(Gd.shape[0]) - Gd * f.ravel()[None, :]
    return sla.solve(A, b.ravel()).reshape(shape)


def forward(op: Operator, f, uin, tol=1e-12, maxiter=1000):
    """Total field u of eq. lipp1 by BiCGStab with the FFT-applied operator."""
    u, it, rr = bicgstab(lambda x: op.A(x, f), uin, tol=tol, maxiter=maxiter)
    return u


# ---------------------------------------------------------------------------
# Data fidelity (eq. prob) and its gradient (Alg. 1 line 6)
# ---------------------------------------------------------------------------

def loss(op: Operator, f, uins, ys, tol=1e-12, weights=None):
    total = 0.0
    for q, (uin, y) in enumerate(zip(uins, ys)):
        u = forward(op, f, uin, tol)
        pred = op.farfield_fft(f * u)
        c = (1.0 / np.vdot(y, y).real) if weights is None else weights[q]
        total += 0.5 * c * np.vdot(pred - y, pred - y).real
    return total


def gradient(op: Operator, f, uins, ys=None, residuals=None, tol=1e-12, weights=None, us=None):
    """sum_q c_q Re(conj(u_q) .* w_q) with (I - G^H diag f) w_q = G~^H r_q.

    This is Re(J_q^H r_q) with J_q = G~ (I - diag(f) G)^{-1} diag(u_q) (the
    Jacobian of eq. lipp2 after the push-through identity), c_q = 1/||y_q||^2
    (eq. prob) unless ``weights`` is given.  ``residuals`` r_q default to
    H_q(f) - y_q.
    """
    g = np.zeros(f.shape, dtype=np.float64)
    for q, uin in enumerate(uins):
        u = forward(op, f, uin, tol) if us is None else us[q]
        if residuals is None:
            r = op.farfield_fft(f * u) - ys[q]
        else:
            r = residuals[q]
        c = (1.0 if ys is None else 1.0 / np.vdot(ys[q], ys[q]).real) if weights is None else weights[q]
        b = op.farfield_adjoint_fft(r)
        w, it, rr = bicgstab(lambda x: op.A(x, f, adjoint=True), b, tol=tol)
        g += c * np.real(np.conj(u) * w)
    return g


def gradient_paper_form(op: Operator, f, u, r):
    """Re(diag(conj u) [G~^H r + G^H (I - diag(f) G^H)^{-1} diag(f) G~^H r]) for one view.

    The form of the Jacobian adjoint with the operator (I - diag(f) G^H) to be
    inverted (Sec. 4.2, with G^H in place of the printed G~^*).
    """
    b = op.farfield_adjoint_fft(r)
    z, it, rr = bicgstab(lambda x: x - f * op.G(x, adjoint=True), f * b, tol=1e-13)
    return np.real(np.conj(u) * (b + op.G(z, adjoint=True)))
