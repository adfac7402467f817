"""Host-side pieces of the reconstruction loop (Sec. 4): FISTA state checkpoints and resumed runs."""
import numpy as np
import torch

from paper_1910_13844_gb300 import recon


def test_fista_state_round_trips(tmp_path):
    f = torch.rand(4, 5, 6)
    st = recon.FistaState(f, f * 2, f * 3, alpha=2.5, k=7, history=[(1, 0.5, 0.1, 0.2)])
    path = str(tmp_path / "state.npz")
    st.save(path)
    back = recon.FistaState.load(path, "cpu")
    assert torch.equal(back.f, st.f) and torch.equal(back.v, st.v) and back.k == 7 and back.alpha == 2.5
    assert np.allclose(back.history[0], st.history[0])


def _stand_ins(monkeypatch):
    # a view-dependent quadratic data term and a positivity-only prox (no library call): enough to make
    # the iterates depend on which views each iteration draws
    gen = torch.Generator().manual_seed(1)
    targets = torch.linspace(0.5, 2.5, 5).reshape(5, 1, 1, 1) * torch.rand(1, 3, 4, 5, generator=gen)

    def data_grad(prob, f, views=None, batched=True, warm=None, stats=None):
        idx = list(range(5)) if views is None else list(views)
        d = f.unsqueeze(0) - targets[idx]
        return 0.5 * float(d.pow(2).sum()), d.sum(dim=0)

    monkeypatch.setattr(recon, "data_grad", data_grad)
    monkeypatch.setitem(recon.PROX, "tv", lambda z, lam, iters: z.clamp_min(0.0))

    class Prob:
        kvec = np.zeros((5, 3))
    return Prob()


def test_resumed_run_draws_the_same_view_subsets(tmp_path, monkeypatch):
    prob = _stand_ins(monkeypatch)
    f0 = torch.zeros(3, 4, 5)
    kw = dict(gamma0=0.1, tau=0.0, subset=2, seed=7)
    full = recon.fista(prob, f0, 10, **kw)
    part = recon.fista(prob, f0, 4, **kw)
    path = str(tmp_path / "fista.npz")
    part.save(path)
    resumed = recon.fista(prob, f0, 6, state=recon.FistaState.load(path, "cpu"), **kw)
    assert resumed.k == full.k == 11
    assert torch.equal(resumed.f, full.f) and torch.equal(resumed.v, full.v)
    # without the saved generator state the resumed run would redraw the first subsets
    stale = recon.FistaState.load(path, "cpu")
    stale.rng = None
    redrawn = recon.fista(prob, f0, 6, state=stale, **kw)
    assert not torch.equal(redrawn.f, full.f)


def test_checkpoint_without_generator_state_still_loads(tmp_path):
    f = torch.rand(2, 2, 2)
    path = str(tmp_path / "old.npz")
    np.savez(path, f=f.numpy(), f_prev=f.numpy(), v=f.numpy(), alpha=1.0, k=3,
             history=np.zeros((0, 4)))
    st = recon.FistaState.load(path, "cpu")
    assert st.rng is None and st.k == 3
