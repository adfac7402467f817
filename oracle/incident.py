"""Incident field from its measurement on the detector plane (Sec. 3.4) and the pupil operator P (Sec. 3.3).

Test infrastructure only.

Sec. 3.4: the 3-D incident field is the free-space propagation of the detector-plane field y_in,
    u_in(., x3) = p_{x3} * y_in,   p_hat_z(w) = exp(-i (x_Gamma - z) sqrt(k_b^2 - |w|^2))   (eq. propUin)
(the square root of k_b^2, not k_b, is taken: the printed kernel has mismatched units).  With
y_in = a exp(i x.k_in) ("tilt transfer", eq. propUin-2) the convolution is applied to the slowly
varying amplitude a with the shifted kernel p_hat_z(w + k_in), then the tilt is multiplied back.
Both convolutions are periodic on the detector grid (the paper computes eq. propUin-2 with a
periodic convolution).  Evanescent components (|w| > k_b) are not propagated (set to zero).

Sec. 3.3: P is a convolution applied by FFT with zero padding to twice the detector size; here
P = crop F^{-1} diag(H) F pad with H(w) = 1{|w| <= k_c} exp(i d sqrt(k_b^2 - |w|^2)) (an ideal
pupil of cut-off k_c followed by a propagation over d, evanescent parts dropped).
"""
from __future__ import annotations

import numpy as np

from .kernel import centred


def detector_coords(m: int, h: float) -> np.ndarray:
    """Pixel centres h (j - m/2 + 1) of one detector axis."""
    return (np.arange(m) - m // 2 + 1) * h


def freqs(m: int, h: float) -> np.ndarray:
    """Angular frequencies of a length-m DFT with pitch h, at storage positions (centred set)."""
    return 2.0 * np.pi * centred(m).astype(np.float64) / (m * h)


def kz(kb: float, wx, wy):
    """sqrt(k_b^2 - |w|^2) and the mask of propagating components."""
    s = kb * kb - wx * wx - wy * wy
    prop = s >= 0.0
    return np.sqrt(np.where(prop, s, 0.0)), prop


def incident_from_detector(y_in: np.ndarray, h: float, kb: float, x_gamma: float, zs: np.ndarray,
                           k_in=None) -> np.ndarray:
    """u_in[z, y, x] for the planes zs from the detector field y_in[y, x] (eqs. propUin, propUin-2).

    k_in = (kx, ky) enables tilt transfer; None propagates y_in directly (the naive method)."""
    my, mx = y_in.shape
    xa, ya = detector_coords(mx, h), detector_coords(my, h)
    wx, wy = np.meshgrid(freqs(mx, h), freqs(my, h))
    if k_in is not None:
        tilt = np.exp(1j * (k_in[0] * xa[None, :] + k_in[1] * ya[:, None]))
        A = np.fft.fft2(y_in * np.conj(tilt))
        sx, sy = wx + k_in[0], wy + k_in[1]
    else:
        tilt = np.ones_like(y_in)
        A = np.fft.fft2(y_in)
        sx, sy = wx, wy
    q, prop = kz(kb, sx, sy)
    out = np.empty((len(zs), my, mx), dtype=np.complex128)
    for i, z in enumerate(zs):
        H = np.where(prop, np.exp(-1j * (x_gamma - z) * q), 0.0)
        out[i] = np.fft.ifft2(A * H) * tilt
    return out


def pupil_transfer(m: tuple, h: float, kb: float, k_cut: float, d: float) -> np.ndarray:
    """H on the 2m-padded detector grid: ideal pupil |w| <= k_cut times propagation over d."""
    My, Mx = 2 * m[0], 2 * m[1]
    wx, wy = np.meshgrid(freqs(Mx, h), freqs(My, h))
    q, prop = kz(kb, wx, wy)
    inside = (wx * wx + wy * wy) <= k_cut * k_cut
    return np.where(prop & inside, np.exp(1j * d * q), 0.0)


def apply_pupil(y: np.ndarray, H: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """P y = crop F^{-1}(H .* F pad(y)) (or P^H with conj(H)); y is placed at offset 0 of the 2m grid."""
    my, mx = y.shape
    pad = np.zeros(H.shape, dtype=np.complex128)
    pad[:my, :mx] = y
    out = np.fft.ifft2((np.conj(H) if adjoint else H) * np.fft.fft2(pad))
    return out[:my, :mx]


def apply_pupil_matrix(y: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Same operator through explicit DFT matrices (no FFT), for small detectors."""
    my, mx = y.shape
    My, Mx = H.shape
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(My), np.arange(My)) / My)
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(Mx), np.arange(Mx)) / Mx)
    pad = np.zeros(H.shape, dtype=np.complex128)
    pad[:my, :mx] = y
    spec = Fy @ pad @ Fx.T
    back = np.conj(Fy) @ (H * spec) @ np.conj(Fx).T / (My * Mx)
    return back[:my, :mx]
