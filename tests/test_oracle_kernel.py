"""Pins of the discrete Green operator (Theorem 1, Proposition 1) in the oracle."""
import numpy as np
import pytest

import phantoms as ph
from oracle import green, kernel

LAM, ETA_B = 0.532, 1.333
KB = green.wavenumber(LAM, ETA_B)
H = LAM / 8


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape,p", [((6, 6, 6), 2), ((6, 6, 6), 4), ((6, 6, 6), 6), ((8, 6, 4), 4)])
def test_prop1_equals_direct_inverse_dft(shape, p):
    # Prop. 1: the sub-lattice sum equals F^{-1}_{np} restricted to Omega_{2n}; the row-column DFT
    # (no FFT) and the FFT restriction are two independent evaluations of the latter.
    a = kernel.kernel_rowcol(shape, H, KB, p)
    b = kernel.kernel_fft(shape, H, KB, p)
    c = kernel.kernel_prop1(shape, H, KB, p)
    assert rel(b, a) < 1e-13
    assert rel(c, a) < 1e-13


def test_prop1_needs_the_centred_index_set(monkeypatch):
    # Planted mistake: DFT index set [-N/2, N/2-1] instead of the centred [-N/2+1, N/2] (Sec. 1.4).
    shape, p = (6, 6, 6), 4
    good = kernel.kernel_prop1(shape, H, KB, p)

    def other(M):
        c = np.arange(M)
        c[c >= M // 2] -= M
        return c

    monkeypatch.setattr(kernel, "centred", other)
    bad = kernel.kernel_prop1(shape, H, KB, p)
    assert rel(bad, good) > 1e-3


def test_theorem1_operator_equals_twofold_padded_convolution():
    shape, p = (8, 6, 4), 4
    v = ph.random_field(shape, 7)
    K = kernel.build_green(shape, H, KB, p)
    Gh = kernel.green_spectrum(K)
    y_thm = kernel.apply_G_theorem1(v, H, KB, p)
    assert rel(kernel.apply_G_fft(Gh, v), y_thm) < 1e-13
    assert rel(kernel.apply_G_direct(K, v), y_thm) < 1e-13
    assert rel(kernel.dense_G(K, shape) @ v.ravel(), y_thm.ravel()) < 1e-13


def test_kernel_and_spectrum_are_even_per_axis():
    shape = (8, 6, 4)
    K = kernel.build_green(shape, H, KB, 4)
    Gh = kernel.green_spectrum(K)
    for ax in range(3):
        flipK = np.roll(np.flip(K, axis=ax), 1, axis=ax)  # value at -d stored at position d
        flipG = np.roll(np.flip(Gh, axis=ax), 1, axis=ax)
        assert np.max(np.abs(flipK - K)) < 1e-13 * np.max(np.abs(K))
        assert np.max(np.abs(flipG - Gh)) < 1e-12 * np.max(np.abs(Gh))


def test_nyquist_entries_never_reach_a_cropped_output():
    # Offsets k - k' of two points of Omega_n lie in [-n+1, n-1]: zeroing the kernel at d = n
    # changes no output of the operator.
    shape = (6, 6, 6)
    raw = kernel.kernel_fft(shape, H, KB, 4)
    v = ph.random_field(shape, 3)
    a = kernel.apply_G_fft(kernel.green_spectrum(raw), v)
    b = kernel.apply_G_fft(kernel.green_spectrum(kernel.zero_nyquist(raw)), v)
    assert rel(a, b) < 1e-13
    assert np.max(np.abs(raw[3])) > 0.0


def test_adjoint_is_convolution_with_conjugate_kernel():
    shape = (8, 6, 4)
    Gh = kernel.green_spectrum(kernel.build_green(shape, H, KB, 4))
    x = ph.random_field(shape, 1)
    y = ph.random_field(shape, 2)
    lhs = np.vdot(y, kernel.apply_G_fft(Gh, x))
    rhs = np.vdot(kernel.apply_G_fft(Gh, y, adjoint=True), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_quadrature_error_falls_with_padding():
    # Theorem 1's bound has a C^tp / p^2 term: with a smooth v the result converges as p grows.
    shape = (8, 8, 8)
    z, y, x = ph.voxel_centres(shape)
    v = np.exp(-(x * x + y * y + z * z) / 4.0) + 0j
    ref = kernel.apply_G_theorem1(v, H, KB, 12)
    errs = [rel(kernel.apply_G_theorem1(v, H, KB, p), ref) for p in (2, 4, 6)]
    assert errs[0] > errs[1] > errs[2]
