"""Pins of the oracle's forward model, far field, solvers and gradient (eqs. lipp1/lipp2, Alg. 1)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import green, kernel, mie, model

LAM, ETA_B = 0.532, 1.333
H = LAM / 8


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def small():
    st = model.setup_from_optics((8, 8, 8), LAM, ETA_B, H)
    op = model.Operator(st)
    f = green.scattering_potential(ph.sphere(st.shape, 3.0, 0.05), ETA_B, LAM)
    uin = model.plane_wave(st.shape, st.h, ph.cone_directions(1, 0.8)[0] * st.kb)
    return st, op, f, uin


def test_farfield_three_ways(small):
    st, op, f, uin = small
    v = ph.random_field(st.shape, 11)
    d = op.farfield_direct(v)
    assert rel(op.farfield_fft(v), d) < 1e-13
    assert rel(op.farfield_matrix() @ v.ravel(), d.ravel()) < 1e-13


def test_farfield_of_a_single_voxel_is_the_green_function(small):
    # one source voxel at centred index (kz, ky, kx) = (1, -2, 3); detector pixel (a, b) at
    # (h (b - m/2 + 1), h (a - m/2 + 1), 3 L/4)
    st, op, f, uin = small
    v = np.zeros(st.shape, dtype=complex)
    n = 8
    v[1 + n // 2 - 1, -2 + n // 2 - 1, 3 + n // 2 - 1] = 2.0 - 1.0j
    y = op.farfield_fft(v)
    a, b = 5, 2
    xd, yd, zd = (b - n // 2 + 1) * H, (a - n // 2 + 1) * H, 0.75 * n * H
    r = np.sqrt((xd - 3 * H) ** 2 + (yd + 2 * H) ** 2 + (zd - H) ** 2)
    assert abs(y[a, b] - H ** 3 * green.green(r, st.kb) * (2.0 - 1.0j)) < 1e-14


def test_farfield_adjoint_dot_product(small):
    st, op, f, uin = small
    v = ph.random_field(st.shape, 12)
    r = ph.random_field(st.det, 13)
    assert abs(np.vdot(r, op.farfield_fft(v)) - np.vdot(op.farfield_adjoint_fft(r), v)) < 1e-12 * np.linalg.norm(r) * np.linalg.norm(v)


def test_bicgstab_matches_dense_lu(small):
    st, op, f, uin = small
    u_lu = model.solve_lu(op, f, uin)
    u_it, it, rr = model.bicgstab(lambda x: op.A(x, f), uin, tol=1e-13)
    assert rel(u_it, u_lu) < 1e-10
    w_lu = model.solve_lu(op, f, uin, adjoint=True)
    w_it, it, rr = model.bicgstab(lambda x: op.A(x, f, adjoint=True), uin, tol=1e-13)
    assert rel(w_it, w_lu) < 1e-10
    # the field actually scatters
    assert rel(u_lu, uin) > 1e-2


def test_zero_potential_gives_incident_field(small):
    st, op, f, uin = small
    zero = np.zeros(st.shape)
    u = model.forward(op, zero, uin)
    assert np.array_equal(u, uin)
    assert np.max(np.abs(op.farfield_fft(zero * u))) == 0.0


def test_born_limit(small):
    # weak contrast: u - u_Born = O(eps^2) while u - u_in = O(eps), with u_Born = u_in + G (f u_in)
    st, op, f, uin = small
    ratios = []
    for eps in (1e-2, 5e-3):
        fe = eps * f
        u = model.solve_lu(op, fe, uin)
        ub = uin + op.G(fe * uin)
        ratios.append(np.linalg.norm(u - ub) / np.linalg.norm(u - uin))
    assert ratios[0] < 0.05
    assert ratios[1] == pytest.approx(ratios[0] / 2, rel=0.05)


def test_reciprocity(small):
    # S = (I - G diag f)^{-1} G is symmetric because the kernel is even: b^T S a = a^T S b
    st, op, f, uin = small
    Gd = kernel.dense_G(op.Kern, st.shape)
    S = np.linalg.solve(np.eye(Gd.shape[0]) - Gd * f.ravel()[None, :], Gd)
    a = ph.random_field(st.shape, 21).ravel()
    b = ph.random_field(st.shape, 22).ravel()
    assert abs(b @ (S @ a) - a @ (S @ b)) < 1e-12 * abs(b @ (S @ a))


def test_gradient_matches_central_differences_and_paper_form(small):
    st, op, f, uin = small
    uins = [uin, model.plane_wave(st.shape, st.h, ph.cone_directions(4, 0.8)[1] * st.kb)]
    noise = [ph.complex_normal(st.det, 5 + q) for q in range(2)]
    ys = [op.farfield_fft(f * model.forward(op, f, u)) + 0.01 * nz * 1e-3 for u, nz in zip(uins, noise)]
    f0 = 0.9 * f
    g = model.gradient(op, f0, uins, ys)
    rng = np.random.default_rng(3)
    d = rng.uniform(-1, 1, st.shape) * (f > 0)
    eps = 1e-3 * np.max(np.abs(f))
    fd = (model.loss(op, f0 + eps * d, uins, ys) - model.loss(op, f0 - eps * d, uins, ys)) / (2 * eps)
    assert np.sum(g * d) == pytest.approx(fd, rel=1e-5)
    # the paper's form (operator (I - diag(f) G^H)) gives the same gradient
    u0 = model.forward(op, f0, uins[0])
    r0 = op.farfield_fft(f0 * u0) - ys[0]
    g0 = model.gradient(op, f0, uins[:1], residuals=[r0], weights=[1.0])
    assert rel(model.gradient_paper_form(op, f0, u0, r0), g0) < 1e-9


def test_mie_coefficients_satisfy_the_optical_theorem():
    # lossless sphere: each partial wave is unitary, |a_l|^2 = -Re a_l
    kb = green.wavenumber(LAM, ETA_B)
    l, a, c = mie.coefficients(0.665, kb, kb * 1.4 / ETA_B)
    assert np.max(np.abs(np.abs(a) ** 2 + a.real)) < 1e-14
    assert np.max(np.abs(a)) > 1e-2


def test_mie_reduces_to_plane_wave_and_is_continuous():
    kb = green.wavenumber(LAM, ETA_B)
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, (3, 50))
    u = mie.total_field(p[0], p[1], p[2], 0.6, kb, kb)
    assert np.max(np.abs(u - np.exp(1j * kb * p[2]))) < 1e-10
    # continuity of u and du/dr across r = a
    k1 = kb * 1.4 / ETA_B
    th = rng.uniform(0, np.pi, 20)
    a = 0.6
    for dr in (1e-7,):
        ri, ro = a - dr, a + dr
        ui = mie.total_field(ri * np.sin(th), 0 * th, ri * np.cos(th), a, kb, k1)
        uo = mie.total_field(ro * np.sin(th), 0 * th, ro * np.cos(th), a, kb, k1)
        assert np.max(np.abs(ui - uo)) < 1e-5
        r2 = 2e-4
        di = (mie.total_field((a - 1e-8) * np.sin(th), 0 * th, (a - 1e-8) * np.cos(th), a, kb, k1)
              - mie.total_field((a - r2) * np.sin(th), 0 * th, (a - r2) * np.cos(th), a, kb, k1)) / (r2 - 1e-8)
        do = (mie.total_field((a + r2) * np.sin(th), 0 * th, (a + r2) * np.cos(th), a, kb, k1)
              - mie.total_field((a + 1e-8) * np.sin(th), 0 * th, (a + 1e-8) * np.cos(th), a, kb, k1)) / (r2 - 1e-8)
        assert np.max(np.abs(di - do)) < 0.02 * np.max(np.abs(di))


def _ls_vs_mie(n, dn=0.02):
    L = 32 * LAM / 8
    rad = 10 * LAM / 8
    h = L / n
    st = model.setup_from_optics((n, n, n), LAM, ETA_B, h)
    op = model.Operator(st)
    f = green.scattering_potential(ph.sphere((n, n, n), rad / h, dn), ETA_B, LAM)
    uin = model.plane_wave(st.shape, h, (0.0, 0.0, st.kb))
    u = model.forward(op, f, uin, tol=1e-10)
    z, y, x = model.coords(st.shape, h)
    k1 = st.kb * (ETA_B + dn) / ETA_B
    um = mie.total_field(x, y, z, rad, st.kb, k1)
    ya, xa, zg = op.detector_points()
    fm = mie.total_field(xa[None, :], ya[:, None], zg, rad, st.kb, k1) - np.exp(1j * st.kb * zg)
    return rel(u - uin, um - uin), rel(op.farfield_fft(f * u), fm)


@pytest.mark.slow
def test_ls_model_converges_to_mie_under_refinement():
    # Sphere of radius 1.25 lambda (10 voxels at h = lambda/8) in a 4 lambda box, sampled at
    # h = lambda/4, lambda/8, lambda/16: the LS error against the analytic field must fall.
    e16 = _ls_vs_mie(16)
    e32 = _ls_vs_mie(32)
    e64 = _ls_vs_mie(64)
    assert e16[0] > e32[0] > e64[0]
    assert e16[1] > e32[1] > e64[1]
    assert e32[0] < 0.05 and e64[0] < 0.015
    assert e64[1] < 5e-3
