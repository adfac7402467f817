"""Pins of the oracle's Green-function pieces (Sec. 2.1, Sec. 3.1) against independent facts."""
import json
import os

import numpy as np
import pytest

from oracle import green

LAM, ETA_B = 0.532, 1.333
KB = green.wavenumber(LAM, ETA_B)
H = LAM / 8
R32 = green.truncation_radius([32 * H] * 3)


def test_wavenumber_and_potential_special_cases():
    # k_b = 2 pi eta_b / lambda; f vanishes for the background and equals k_b^2 when eta^2 = 2 eta_b^2
    assert KB == pytest.approx(2 * np.pi * 1.333 / 0.532, rel=1e-15)
    assert green.scattering_potential(np.array([0.0]), ETA_B, LAM)[0] == 0.0
    dn = ETA_B * (np.sqrt(2.0) - 1.0)
    assert green.scattering_potential(np.array([dn]), ETA_B, LAM)[0] == pytest.approx(KB * KB, rel=1e-12)


def test_green_solves_helmholtz_and_is_outgoing():
    # (Laplace + k^2) g = 0 away from 0, checked with a 4th-order radial finite difference of r g;
    # outgoing: r (dg/dr - i k g) -> 0.
    r = np.linspace(1.0, 3.0, 9)
    dr = 1e-3
    rg = lambda rr: rr * green.green(rr, KB)
    d2 = (-rg(r + 2 * dr) + 16 * rg(r + dr) - 30 * rg(r) + 16 * rg(r - dr) - rg(r - 2 * dr)) / (12 * dr * dr)
    lap = d2 / r
    assert np.max(np.abs(lap + KB * KB * green.green(r, KB))) < 1e-6 * KB * KB * np.max(np.abs(green.green(r, KB)))
    big = np.array([1e3, 1e4])
    dg = (green.green(big + 1e-4, KB) - green.green(big - 1e-4, KB)) / 2e-4
    assert np.all(np.abs(big * (dg - 1j * KB * green.green(big, KB))) < 2e-3)


@pytest.mark.parametrize("scale", [0.0, 0.1, 0.5, 0.99, 1.0 - 1e-7, 1.0, 1.0 + 1e-6, 1.01, 1.7, 3.0])
def test_ghat_closed_form_matches_quadrature(scale):
    w = scale * KB
    closed = green.ghat_t(np.array([w]), KB, R32)[0]
    quad = green.ghat_t_quadrature(np.array([w]), KB, R32, nodes=8192)[0]
    assert abs(closed - quad) <= 1e-9 * abs(quad)


def test_ghat_at_zero_is_integral_over_ball():
    assert abs(green.ghat_t(np.array([0.0]), KB, R32)[0] - green.ghat_t_zero(KB, R32)) < 1e-13 * abs(green.ghat_t_zero(KB, R32))


def test_greenL2_is_the_continuous_extension():
    # eq. GreenL2 at ||w|| = k_b is the limit of eq. GreenL from both sides
    at = green.ghat_t(np.array([KB]), KB, R32)[0]
    for eps in (1e-4, 1e-5):
        for s in (-1, 1):
            near = green.ghat_t(np.array([KB * (1 + s * eps)]), KB, R32)[0]
            assert abs(near - at) < 50 * eps * KB * R32 * abs(at)


def test_golden_quadrature_values():
    with open(os.path.join(os.path.dirname(__file__), "golden", "ghat_t_quadrature.json")) as fh:
        gold = json.load(fh)
    vals = green.ghat_t(np.array(gold["w"]), gold["kb"], gold["R"])
    ref = np.array(gold["re"]) + 1j * np.array(gold["im"])
    assert np.max(np.abs(vals - ref) / np.abs(ref)) < 1e-9


def test_printed_sinc_sign_is_rejected_by_the_pin():
    # Planted mistake: the sign as printed in eq. GreenL.  It puts a pole at ||w|| = k_b and
    # breaks the value at 0; the quadrature pin must catch it.
    ws = np.array([0.0, 0.5 * KB, 1.5 * KB])
    wrong = green.ghat_t(ws, KB, R32, _sinc_sign=+1.0)
    quad = green.ghat_t_quadrature(ws, KB, R32)
    assert np.min(np.abs(wrong - quad) / np.abs(quad)) > 1e-2
    near = green.ghat_t(np.array([KB * (1 + 1e-9)]), KB, R32, _sinc_sign=+1.0)[0]
    assert abs(near) > 1e6 * abs(green.ghat_t(np.array([KB]), KB, R32)[0])


def test_fig3_workload_satisfies_theorem1_sampling_condition():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_fig3.json")) as fh:
        fig = json.load(fh)
    lam = fig["lambda_nm"] * 1e-3
    h = fig["h_over_lambda"] * lam
    L = fig["n"] * h
    kb = green.wavenumber(lam, fig["eta_b"])
    # Theorem 1 requires n > k_b L / pi  (equivalently k_b < pi / h)
    assert fig["n"] > kb * L / np.pi
    assert kb < np.pi / h
    # the bead (diameter 3 lambda) fits inside Omega = [-L/2, L/2]^3
    assert 3 * lam < L
