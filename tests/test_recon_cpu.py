"""Host-side pieces of the reconstruction loop (Sec. 4): FISTA state checkpoints."""
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
