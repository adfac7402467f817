"""Discrete Green operator G of Theorem 1 and the kernel of Proposition 1 (oracle).

Conventions (Sec. 1.4, Theorem 1, eq. padV):
* a length-M axis uses the centred index set [-M/2+1, M/2]; centred index c is
  stored at array position c mod M, so numpy's fft/ifft are the paper's F and
  F^{-1} (both are M-periodic in the index);
* a volume array ``v[z, y, x]`` of shape (nz, ny, nx) holds the sample with
  centred index (i - n/2 + 1) at array position i;
* L_i = n_i h, the sampling step of the Green spectrum is delta_i = 2 pi / (p L_i).

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .green import ghat_t, truncation_radius

_WORKERS = -1


def centred(M: int) -> np.ndarray:
    """Centred index held at each storage position 0..M-1 (Sec. 1.4)."""
    c = np.arange(M)
    c[c > M // 2] -= M
    return c


def _embed(v: np.ndarray, M) -> np.ndarray:
    """Place v (array positions i, centred i - n/2 + 1) on an M grid at positions (c mod M) (eq. padV)."""
    out = np.zeros(tuple(M), dtype=np.complex128)
    idx = [((np.arange(n) - n // 2 + 1) % m) for n, m in zip(v.shape, M)]
    out[np.ix_(*idx)] = v
    return out


def _extract(a: np.ndarray, shape) -> np.ndarray:
    """Inverse of ``_embed``: read the entries of the centred set Omega_n (Remark 1's crop)."""
    idx = [((np.arange(n) - n // 2 + 1) % m) for n, m in zip(shape, a.shape)]
    return a[np.ix_(*idx)]


def ghat_samples(shape_n, h: float, kb: float, p: int) -> np.ndarray:
    """ghat_t(delta q) for q in Omega_{np} (Theorem 1), at storage positions q mod np."""
    shape_n = tuple(int(s) for s in shape_n)
    R = truncation_radius([s * h for s in shape_n])
    axes = []
    for n in shape_n:
        delta = 2.0 * np.pi / (p * n * h)
        axes.append(delta * centred(n * p).astype(np.float64))

    wz, wy, wx = np.meshgrid(*axes, indexing="ij")
    w = np.sqrt(wz * wz + wy * wy + wx * wx)
    return ghat_t(w, kb, R)


def apply_G_theorem1(v: np.ndarray, h: float, kb: float, p: int = 4) -> np.ndarray:
    """(G v)[k] = (F^{-1}(ghat_t(delta q) .* F v_p))[k] for k in Omega_n (Theorem 1, Remark 1).

    v_p is v zero-padded p times on the centred grid (eq. padV).  This is the
    definition of the discrete operator; it costs (np)^3 memory.
    """
    M = [s * p for s in v.shape]
    vp = _embed(v, M)
    gh = ghat_samples(v.shape, h, kb, p)
    y = sfft.ifftn(gh * sfft.fftn(vp, workers=_WORKERS), workers=_WORKERS)
    return _extract(y, v.shape)


def kernel_rowcol(shape_n, h: float, kb: float, p: int = 4) -> np.ndarray:
    """K[d] = (np)^{-3} sum_{q in Omega_np} ghat_t(delta q) e^{2 i pi q.d/(np)}, d in Omega_{2n}.

    Written as an explicit inverse DFT, one axis at a time with dense DFT
    matrices (no FFT).  Returned at storage positions d mod 2n.  This is the
    right-hand side of Proposition 1 written directly as F^{-1}_{np} restricted
    to Omega_{2n} (proof of Prop. 1).  Cost O((np)^4); small grids only.
    """
    shape_n = tuple(int(s) for s in shape_n)
    t = ghat_samples(shape_n, h, kb, p)
    for ax, n in enumerate(shape_n):
        q = centred(n * p).astype(np.float64)
        d = centred(2 * n).astype(np.float64)
        E = np.exp(2j * np.pi * np.outer(d, q) / (n * p)) / (n * p)
        t = np.moveaxis(np.tensordot(t, E, axes=([ax], [1])), -1, ax)
    return t


def kernel_fft(shape_n, h: float, kb: float, p: int = 4) -> np.ndarray:
    """Same K as ``kernel_rowcol`` through one inverse FFT on the np grid, then restriction to Omega_{2n}."""
    shape_n = tuple(int(s) for s in shape_n)
    t = sfft.ifftn(ghat_samples(shape_n, h, kb, p), workers=_WORKERS)
    idx = [centred(2 * n) % (n * p) for n in shape_n]
    return t[np.ix_(*idx)]


def kernel_prop1(shape_n, h: float, kb: float, p: int = 4) -> np.ndarray:
    """Modified kernel g_t^m of Proposition 1 on Omega_{2n}:

        g^m[k] = (8/p^3) sum_{s in [0, p/2-1]^3} F^{-1}_{2n}(ghat_t[(p/2) . - s])[k] e^{-2 i pi k.s/(np)}

    Each sub-lattice sample ghat_t[(p/2) q - s], q in Omega_{2n}, is the value
    of ghat_t at frequency delta ((p/2) q - s).  Returned at storage positions
    k mod 2n.
    """
    assert p % 2 == 0 and p >= 2
    shape_n = tuple(int(s) for s in shape_n)
    R = truncation_radius([s * h for s in shape_n])
    half = p // 2
    out = np.zeros(tuple(2 * n for n in shape_n), dtype=np.complex128)
    qs = [centred(2 * n).astype(np.float64) for n in shape_n]
    ks = qs
    deltas = [2.0 * np.pi / (p * n * h) for n in shape_n]
    for sz in range(half):
        for sy in range(half):
            for sx in range(half):
                s = (sz, sy, sx)
                comps = [d * (half * q - si) for d, q, si in zip(deltas, qs, s)]
                wz, wy, wx = np.meshgrid(*comps, indexing="ij")
                sub = ghat_t(np.sqrt(wz * wz + wy * wy + wx * wx), kb, R)
                t = sfft.ifftn(sub, workers=_WORKERS)
                ph = [np.exp(-2j * np.pi * k * si / (n * p)) for k, si, n in zip(ks, s, shape_n)]
                out += t * ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
    return out * (8.0 / p ** 3)


def zero_nyquist(K: np.ndarray) -> np.ndarray:
    """Set the kernel to 0 at the Nyquist offset d_i = n_i of each axis of the 2n grid.

    Offsets k - k' of two points of Omega_n lie in [-n+1, n-1], so d = n never
    reaches a cropped output.  Fixing it to zero makes the stored spectrum a
    function of the cropped operator alone.
    """
    K = K.copy()
    nz, ny, nx = (s // 2 for s in K.shape)
    K[nz, :, :] = 0.0
    K[:, ny, :] = 0.0
    K[:, :, nx] = 0.0
    return K


def green_spectrum(K: np.ndarray) -> np.ndarray:
    """Spectrum of the reduced-padding kernel on the 2n grid: F_{2n}(K) (Prop. 1)."""
    return sfft.fftn(K, workers=_WORKERS)


def build_green(shape_n, h: float, kb: float, p: int = 4, method: str = "fft") -> np.ndarray:
    """Kernel K on Omega_{2n} with Nyquist offsets zeroed, computed by the named method."""
    fn = {"fft": kernel_fft, "rowcol": kernel_rowcol, "prop1": kernel_prop1}[method]
    return zero_nyquist(fn(shape_n, h, kb, p))


def apply_G_direct(K: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(G v)[k] = sum_{k' in Omega_n} K[k - k'] v[k'] by direct summation (brute force, tiny grids)."""
    nz, ny, nx = v.shape
    Mz, My, Mx = K.shape
    out = np.zeros(v.shape, dtype=np.complex128)
    iz, iy, ix = np.arange(nz), np.arange(ny), np.arange(nx)
    for a in range(nz):
        dz = (a - iz) % Mz
        for b in range(ny):
            dy = (b - iy) % My
            for c in range(nx):
                dx = (c - ix) % Mx
                out[a, b, c] = np.sum(K[np.ix_(dz, dy, dx)] * v)
    return out


def apply_G_fft(Ghat: np.ndarray, v: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """G v (or G^H v) with twofold padding: crop(F^{-1}(Ghat .* F v_2)) (Prop. 1).

    G^H is the convolution with conj(K); since K is even its spectrum is conj(Ghat).
    """
    vp = _embed(v, Ghat.shape)
    spec = np.conj(Ghat) if adjoint else Ghat
    y = sfft.ifftn(spec * sfft.fftn(vp, workers=_WORKERS), workers=_WORKERS)
    return _extract(y, v.shape)


def dense_G(K: np.ndarray, shape) -> np.ndarray:
    """Explicit N x N matrix G[k, k'] = K[k - k'] (rows/cols in C order of ``shape``); tiny grids."""
    nz, ny, nx = shape
    Mz, My, Mx = K.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    dz = (z[:, None] - z[None, :]) % Mz
    dy = (y[:, None] - y[None, :]) % My
    dx = (x[:, None] - x[None, :]) % Mx
    return K[dz, dy, dx]
