"""GPU Green spectrum and FFT-convolution operator vs the FP64 oracle (Theorem 1, Prop. 1)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import kernel, model

from gpu_common import H, KB, potential, rel, to_dev, torch_and_lib

# (nz, ny, nx): cubic, non-cubic with ragged CTA tiles (2nx = 24, 48; rows not a multiple of the tile),
# and a config-sized non-cubic grid
SHAPES = [(8, 8, 8), (12, 16, 24), (16, 8, 12), (32, 32, 32), (24, 48, 16), (96, 128, 128)]
# every z transform length of the pass table: 96 and 384 run the TMA-staged z pass with their own
# split (16 x 6; 32 x 12 on 16 threads per column), 144 and 288 the column-group one
Z_LENGTHS = [(48, 24, 16), (192, 16, 16), (72, 16, 16), (144, 16, 32)]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", SHAPES[:5])
def test_green_spectrum_matches_oracle(shape):
    torch, ls = torch_and_lib()
    nz, ny, nx = shape
    plan = ls.Plan(shape, KB, H)
    full = torch.empty((2 * nz, 2 * ny, 2 * nx), dtype=torch.complex64, device="cuda")
    ls.ls_green_spectrum(plan.handle, 4, full)
    torch.cuda.synchronize()
    ref = kernel.green_spectrum(kernel.build_green(shape, H, KB, 4))
    got = full.cpu().numpy()
    assert rel(got, ref) < 2e-6
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", SHAPES + Z_LENGTHS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_green_operator_and_matvec_match_oracle(shape, adjoint):
    torch, ls = torch_and_lib()
    plan = ls.Plan(shape, KB, H)
    v = ph.random_field(shape, 5)
    dn = ph.random_ellipsoids(shape, count=4, rmin=2, rmax=max(3, min(shape) // 4))
    f = potential(dn)
    Gh = kernel.green_spectrum(kernel.build_green(shape, H, KB, 4))
    vd = to_dev(torch, v, torch.complex64)
    fd = to_dev(torch, f, torch.float32)
    out = torch.empty_like(vd)
    ls.ls_apply_green(plan.handle, vd, out, adjoint)
    torch.cuda.synchronize()
    ref = kernel.apply_G_fft(Gh, vd.cpu().numpy().astype(np.complex128), adjoint)
    assert rel(out.cpu().numpy(), ref) < 1e-5
    y = torch.empty_like(vd)
    ls.ls_matvec(plan.handle, fd, vd, y, adjoint)
    torch.cuda.synchronize()
    x64 = vd.cpu().numpy().astype(np.complex128)
    f32 = fd.cpu().numpy().astype(np.float64)
    ref = x64 - kernel.apply_G_fft(Gh, f32 * x64, adjoint)
    assert rel(y.cpu().numpy(), ref) < 1e-5
    plan.close()


# every form of the TMA-staged z pass (split, persistence) on a batch of views, forced through an
# autotune cache entry: 96-point (16 x 6), 384-point (32 x 12 on 16 threads per column, two stage-2
# sub-transforms per thread) and 64-point transforms
Z_FORMS = [(0, 0), (0, 1), (0, 2), (1, 0)]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(48, 24, 16), (192, 16, 16), (32, 16, 48)])
@pytest.mark.parametrize("form", Z_FORMS)
def test_every_z_pass_form_matches_oracle_on_a_batch(tmp_path, monkeypatch, shape, form):
    torch, ls = torch_and_lib()
    split, persist = form
    nz, ny, nx = shape
    q = 3
    cache = tmp_path / "tune.txt"
    key = f"{torch.cuda.get_device_name().replace(' ', '_')}:{nx}x{ny}x{nz}:{q}"
    cache.write_text(f"{key} 1 1 0 2 1 1.0 1.0 {split} 0 0 {persist} 0\n")
    monkeypatch.setenv("LS_AUTOTUNE_CACHE", str(cache))
    f = potential(ph.random_ellipsoids(shape, count=4, rmin=2, rmax=max(3, min(shape) // 4)))
    fd = to_dev(torch, f, torch.float32)
    plan = ls.Plan(shape, KB, H)
    t = plan.autotune(q, fd)
    assert t["from_cache"] == 1 and t["z_persist"] == persist
    x = torch.stack([to_dev(torch, ph.random_field(shape, 10 + i), torch.complex64) for i in range(q)])
    Gh = kernel.green_spectrum(kernel.build_green(shape, H, KB, 4))
    f32 = fd.cpu().numpy().astype(np.float64)
    for adjoint in (False, True):
        y = torch.empty_like(x)
        ls.ls_matvec_batch(plan.handle, fd, x, y, adjoint)
        torch.cuda.synchronize()
        for i in range(q):
            x64 = x[i].cpu().numpy().astype(np.complex128)
            ref = x64 - kernel.apply_G_fft(Gh, f32 * x64, adjoint)
            assert rel(y[i].cpu().numpy(), ref) < 1e-5, (form, adjoint, i)
    plan.close()


@pytest.mark.gpu
def test_operator_is_deterministic_and_linear():
    torch, ls = torch_and_lib()
    shape = (16, 16, 16)
    plan = ls.Plan(shape, KB, H)
    a = to_dev(torch, ph.random_field(shape, 1), torch.complex64)
    b = to_dev(torch, ph.random_field(shape, 2), torch.complex64)
    ga, gb, gab, gab2 = (torch.empty_like(a) for _ in range(4))
    ls.ls_apply_green(plan.handle, a, ga)
    ls.ls_apply_green(plan.handle, b, gb)
    ls.ls_apply_green(plan.handle, a + 2 * b, gab)
    ls.ls_apply_green(plan.handle, a + 2 * b, gab2)
    torch.cuda.synchronize()
    assert torch.equal(gab, gab2)
    assert rel((ga + 2 * gb).cpu().numpy(), gab.cpu().numpy()) < 1e-6
    # adjoint dot-product test <G a, b> = <a, G^H b>
    gha = torch.empty_like(a)
    ls.ls_apply_green(plan.handle, b, gha, True)
    torch.cuda.synchronize()
    lhs = np.vdot(b.cpu().numpy(), ga.cpu().numpy())
    rhs = np.vdot(gha.cpu().numpy(), a.cpu().numpy())
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    plan.close()


@pytest.mark.gpu
def test_batched_matvec_equals_single_matvecs():
    torch, ls = torch_and_lib()
    shape = (12, 16, 24)
    plan = ls.Plan(shape, KB, H)
    f = to_dev(torch, potential(ph.random_ellipsoids(shape, count=3, rmin=2, rmax=4)), torch.float32)
    x = torch.stack([to_dev(torch, ph.random_field(shape, 60 + q), torch.complex64) for q in range(5)])
    y = torch.empty_like(x)
    ls.ls_matvec_batch(plan.handle, f, x, y, True)
    for q in range(5):
        yq = torch.empty_like(x[q])
        ls.ls_matvec(plan.handle, f, x[q], yq, True)
        torch.cuda.synchronize()
        assert torch.equal(yq, y[q])
    plan.close()
