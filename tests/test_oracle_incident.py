"""Pins of the incident-field propagation with tilt transfer (Sec. 3.4, Fig. 4) and of the pupil operator P."""
import numpy as np
import pytest

import phantoms as ph
from oracle import green, incident

LAM, ETA_B, H = ph.LAMBDA_UM, ph.ETA_B, ph.VOXEL_UM
KB = green.wavenumber(LAM, ETA_B)


def _tilted_wave(m, kvec, z):
    xa = incident.detector_coords(m, H)
    return np.exp(1j * (kvec[0] * xa[None, :] + kvec[1] * xa[:, None] + kvec[2] * z))


@pytest.mark.parametrize("q", [0, 7, 23])
def test_tilt_transfer_reproduces_a_tilted_plane_wave_exactly(q):
    # a plane wave with an arbitrary (off-grid) tilt, measured on the detector, propagated back into
    # the volume: with tilt transfer the amplitude is constant and the result is exact (Fig. 4)
    m, nz = 32, 32
    x_gamma = 0.75 * nz * H
    k = ph.cone_directions(40, 0.8)[q] * KB
    y_in = _tilted_wave(m, k, x_gamma)
    zs = (np.arange(nz) - nz // 2 + 1) * H
    u = incident.incident_from_detector(y_in, H, KB, x_gamma, zs, k_in=k[:2])
    exact = np.stack([_tilted_wave(m, k, z) for z in zs])
    assert np.max(np.abs(u - exact)) < 1e-12


def test_naive_propagation_is_worse_for_off_grid_tilts():
    m, nz = 32, 32
    x_gamma = 0.75 * nz * H
    k = ph.cone_directions(40, 0.8)[7] * KB
    y_in = _tilted_wave(m, k, x_gamma)
    zs = (np.arange(nz) - nz // 2 + 1) * H
    exact = np.stack([_tilted_wave(m, k, z) for z in zs])
    naive = incident.incident_from_detector(y_in, H, KB, x_gamma, zs, k_in=None)
    assert np.linalg.norm(naive - exact) / np.linalg.norm(exact) > 1e-2


def test_propagation_to_the_detector_plane_is_the_identity_on_band_limited_fields():
    m = 16
    x_gamma = 1.0
    rng = np.random.default_rng(0)
    spec = np.zeros((m, m), dtype=complex)
    wx, wy = np.meshgrid(incident.freqs(m, H), incident.freqs(m, H))
    inside = wx * wx + wy * wy < 0.8 * KB * KB
    spec[inside] = rng.standard_normal(inside.sum()) + 1j * rng.standard_normal(inside.sum())
    y = np.fft.ifft2(spec)
    u = incident.incident_from_detector(y, H, KB, x_gamma, np.array([x_gamma]))
    assert np.max(np.abs(u[0] - y)) < 1e-13


def test_pupil_operator_definition_adjoint_and_semigroup():
    m = (12, 10)
    kc = 0.6 * KB
    H1 = incident.pupil_transfer(m, H, KB, kc, 0.4)
    y = ph.random_field(m, 3)
    r = ph.random_field(m, 4)
    assert np.allclose(incident.apply_pupil(y, H1), incident.apply_pupil_matrix(y, H1), atol=1e-12)
    lhs = np.vdot(r, incident.apply_pupil(y, H1))
    rhs = np.vdot(incident.apply_pupil(r, H1, adjoint=True), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # propagation over d1 then d2 equals propagation over d1 + d2 on the padded grid (no crop)
    Ha = incident.pupil_transfer(m, H, KB, 10 * KB, 0.3)
    Hb = incident.pupil_transfer(m, H, KB, 10 * KB, 0.5)
    Hab = incident.pupil_transfer(m, H, KB, 10 * KB, 0.8)
    prop = np.abs(Hab) > 0
    assert np.allclose((Ha * Hb)[prop], Hab[prop], atol=1e-13)
    # d = 0 with an open pupil keeps every propagating component
    H0 = incident.pupil_transfer(m, H, KB, 10 * KB, 0.0)
    assert set(np.unique(np.abs(H0)).round(12)) <= {0.0, 1.0}
