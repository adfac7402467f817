"""Helpers shared by the GPU parity tests (inputs from phantoms/, expectations from oracle/)."""
import numpy as np
import pytest

import phantoms as ph
from oracle import green, model

LAM, ETA_B, H = ph.LAMBDA_UM, ph.ETA_B, ph.VOXEL_UM
KB = green.wavenumber(LAM, ETA_B)


def torch_and_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_13844_gb300 as ls

    return torch, ls


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def potential(dn):
    return green.scattering_potential(dn, ETA_B, LAM)
