"""Host-side pieces of the reconstruction loop (Sec. 4): TV prox by FGP and FISTA state checkpoints."""
import numpy as np
import torch

from paper_1910_13844_gb300 import recon


def test_grad_and_div_are_negative_adjoints():
    g = torch.Generator().manual_seed(1)
    a = torch.randn(5, 6, 7, dtype=torch.float64, generator=g)
    p = torch.randn(3, 5, 6, 7, dtype=torch.float64, generator=g)
    assert abs(float((recon._grad3(a) * p).sum() + (a * recon._div3(p)).sum())) < 1e-10


def test_tv_prox_is_a_constrained_minimiser():
    g = torch.Generator().manual_seed(0)
    z = torch.randn(8, 9, 10, dtype=torch.float64, generator=g)
    lam = 0.3
    x = recon.prox_tv_nonneg(z, lam, 2000)

    def obj(v):
        return 0.5 * ((v - z) ** 2).sum() + lam * recon._grad3(v).pow(2).sum(0).sqrt().sum()

    assert float(x.min()) >= 0.0
    best = float(obj(x))
    for _ in range(100):
        y = (x + 1e-3 * torch.randn(x.shape, dtype=x.dtype, generator=g)).clamp_min(0)
        assert float(obj(y)) >= best - 1e-7
    # lam = 0 is the projection on the non-negative orthant
    assert torch.equal(recon.prox_tv_nonneg(z, 0.0), z.clamp_min(0.0))


def test_fista_state_round_trips(tmp_path):
    f = torch.rand(4, 5, 6)
    st = recon.FistaState(f, f * 2, f * 3, alpha=2.5, k=7, history=[(1, 0.5, 0.1, 0.2)])
    path = str(tmp_path / "state.npz")
    st.save(path)
    back = recon.FistaState.load(path, "cpu")
    assert torch.equal(back.f, st.f) and torch.equal(back.v, st.v) and back.k == 7 and back.alpha == 2.5
    assert np.allclose(back.history[0], st.history[0])
