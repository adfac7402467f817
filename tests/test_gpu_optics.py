"""GPU incident-field propagation (Sec. 3.4, eqs. propUin / propUin-2) and pupil operator P (Sec. 3.3)
against the FP64 oracle, and P inside the forward model and gradient (eq. lipp2)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import incident, model

from gpu_common import ETA_B, H, KB, LAM, potential, rel, to_dev, torch_and_lib


def _tilted_wave(my, mx, kvec, z):
    xa, ya = incident.detector_coords(mx, H), incident.detector_coords(my, H)
    return np.exp(1j * (kvec[0] * xa[None, :] + kvec[1] * ya[:, None] + kvec[2] * z))


def _band_limited(my, mx, seed, frac=0.7):
    rng = np.random.default_rng(seed)
    wx, wy = np.meshgrid(incident.freqs(mx, H), incident.freqs(my, H))
    inside = wx * wx + wy * wy < frac * KB * KB
    spec = np.zeros((my, mx), dtype=complex)
    spec[inside] = rng.standard_normal(inside.sum()) + 1j * rng.standard_normal(inside.sum())
    y = np.fft.ifft2(spec)
    return y / np.max(np.abs(y))


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 12, 16)])
@pytest.mark.parametrize("tilt", [False, True])
def test_incident_field_matches_oracle(shape, tilt):
    torch, ls = torch_and_lib()
    nz, ny, nx = shape
    plan = ls.Plan(shape, KB, H)
    x_gamma = 0.75 * nz * H
    kvecs = ph.cone_directions(3, 0.8) * KB
    zs = (np.arange(nz) - nz // 2 + 1) * H
    ys = []
    for q, k in enumerate(kvecs):
        # a tilted wave times a smooth band-limited envelope, as measured without a sample
        ys.append(_tilted_wave(ny, nx, k, x_gamma) * (1.0 + 0.3 * _band_limited(ny, nx, 70 + q, 0.05)))
    yd = torch.stack([to_dev(torch, y, torch.complex64) for y in ys])
    u = plan.field(3)
    ls.ls_incident_field(plan.handle, yd, u, k_in=kvecs[:, :2] if tilt else None)
    torch.cuda.synchronize()
    for q, k in enumerate(kvecs):
        y32 = yd[q].cpu().numpy().astype(np.complex128)
        ref = incident.incident_from_detector(y32, H, KB, x_gamma, zs, k_in=k[:2] if tilt else None)
        assert rel(u[q].cpu().numpy(), ref) < 1e-5
    plan.close()


@pytest.mark.gpu
def test_tilt_transfer_on_gpu_recovers_the_plane_wave():
    # off-grid tilt: propagating the measured plane wave reproduces the plane wave inside the volume
    torch, ls = torch_and_lib()
    shape = (32, 32, 32)
    plan = ls.Plan(shape, KB, H)
    x_gamma = 0.75 * 32 * H
    k = ph.cone_directions(40, 0.8)[7] * KB
    y = to_dev(torch, _tilted_wave(32, 32, k, x_gamma)[None], torch.complex64)
    u = plan.field(1)
    ls.ls_incident_field(plan.handle, y, u, k_in=k[None, :2])
    ref = plan.plane_waves(k[None])
    torch.cuda.synchronize()
    assert rel(u.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,det", [((16, 16, 16), None), ((12, 24, 16), (18, 12))])
def test_pupil_matches_oracle_and_is_adjoint(shape, det):
    torch, ls = torch_and_lib()
    opts = {} if det is None else {"det_my": det[0], "det_mx": det[1]}
    plan = ls.Plan(shape, KB, H, **opts)
    kc, d = 0.6 * KB, -0.9
    ls.ls_set_pupil(plan.handle, kc, d)
    Hd = incident.pupil_transfer(plan.det, H, KB, kc, d)
    y = torch.stack([to_dev(torch, ph.random_field(plan.det, 50 + q), torch.complex64) for q in range(2)])
    r = torch.stack([to_dev(torch, ph.random_field(plan.det, 60 + q), torch.complex64) for q in range(2)])
    py, phr = torch.empty_like(y), torch.empty_like(r)
    ls.ls_apply_pupil(plan.handle, y, py)
    ls.ls_apply_pupil(plan.handle, r, phr, adjoint=True)
    torch.cuda.synchronize()
    for q in range(2):
        yq = y[q].cpu().numpy().astype(np.complex128)
        rq = r[q].cpu().numpy().astype(np.complex128)
        assert rel(py[q].cpu().numpy(), incident.apply_pupil(yq, Hd)) < 1e-5
        assert rel(phr[q].cpu().numpy(), incident.apply_pupil(rq, Hd, adjoint=True)) < 1e-5
        lhs = np.vdot(rq, py[q].cpu().numpy().astype(np.complex128))
        rhs = np.vdot(phr[q].cpu().numpy().astype(np.complex128), yq)
        assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    # in-place application
    z = y.clone()
    ls.ls_apply_pupil(plan.handle, z, z)
    torch.cuda.synchronize()
    assert torch.equal(z, py)
    plan.close()


@pytest.mark.gpu
def test_forward_and_gradient_with_pupil_match_oracle():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    st = model.setup_from_optics(shape, LAM, ETA_B, H)
    op = model.Operator(st)
    f_true = potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=5, dn_max=0.05))
    kvecs = ph.cone_directions(2, 0.8) * KB
    kc, d = 0.7 * KB, -st.zgamma
    Hd = incident.pupil_transfer(st.det, H, KB, kc, d)
    uins = [model.plane_wave(shape, H, k) for k in kvecs]
    ys = []
    for q, u0 in enumerate(uins):
        u = model.forward(op, f_true, u0, tol=1e-12)
        ys.append(incident.apply_pupil(op.farfield_fft(f_true * u), Hd) + 0.01 * ph.complex_normal(st.det, 90 + q))
    plan = ls.Plan(shape, KB, H, tol=1e-7)
    ls.ls_set_pupil(plan.handle, kc, d)
    f0 = 0.9 * f_true
    f = to_dev(torch, f0, torch.float32)
    uin = plan.plane_waves(kvecs)
    u, far, code, _ = plan.forward(f, uin)
    torch.cuda.synchronize()
    assert code == ls.LS_OK
    f032 = f.cpu().numpy().astype(np.float64)
    for q, u0 in enumerate(uins):
        uq = model.forward(op, f032, u0, tol=1e-12)
        assert rel(far[q].cpu().numpy(), incident.apply_pupil(op.farfield_fft(f032 * uq), Hd)) < 1e-4
    y = torch.stack([to_dev(torch, x, torch.complex64) for x in ys])
    res = torch.empty_like(far)
    ls.ls_residual(far, y, res)
    g, code, stats = plan.gradient(f, res, u_fwd=u)
    torch.cuda.synchronize()
    assert code == ls.LS_OK, stats
    # oracle gradient of sum_q 1/2 ||P G~(f u_q) - y_q||^2: adjoint right-hand side G~^H P^H r
    us = [model.forward(op, f032, u0, tol=1e-12) for u0 in uins]
    rs = [incident.apply_pupil(op.farfield_fft(f032 * uq), Hd) - yq for uq, yq in zip(us, ys)]
    g_ref = model.gradient(op, f032, uins, residuals=[incident.apply_pupil(r, Hd, adjoint=True) for r in rs],
                           weights=[1.0, 1.0], us=us, tol=1e-12)
    assert rel(g.cpu().numpy(), g_ref) < 1e-3
    # removing the pupil restores the plain model
    ls.ls_set_pupil(plan.handle, 0.0, 0.0)
    _, far0, _, _ = plan.forward(f, uin)
    torch.cuda.synchronize()
    uq = model.forward(op, f032, uins[0], tol=1e-12)
    assert rel(far0[0].cpu().numpy(), op.farfield_fft(f032 * uq)) < 1e-4
    plan.close()


@pytest.mark.gpu
def test_pupil_rejects_a_padded_detector_without_fft_length():
    torch, ls = torch_and_lib()
    plan = ls.Plan((12, 24, 16), KB, H, det_my=20, det_mx=12)  # 2 m_y = 40 = 2^3 5
    with pytest.raises(ls.LsError) as e:
        ls.ls_set_pupil(plan.handle, 0.5 * KB, 0.0)
    assert e.value.code == ls.LS_EUNSUPPORTED
    plan.close()
