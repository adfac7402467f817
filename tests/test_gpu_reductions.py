"""Sums across threads in the solver's reductions are float64.

The solver's inner products and norms (the BiCGStab scalars of Sec. 2.2) are float32 products with
per-thread float32 partial sums, then one float64 sum across the threads of a block (warp shuffles
included) and float64 above.  These tests build inputs for which each thread holds exactly one
exactly-representable term, so the float64 result is exact, while a float32 sum across the 32
lanes of a warp (simulated below on the host, shuffle by shuffle) loses low-order bits: a
cancelling inner product through ls_inner_products, and a norm through ls_residual (the same
reduction helper as the solver's kernels).
"""
import numpy as np
import pytest

from gpu_common import torch_and_lib

COUNT = 64 * 256   # 64 blocks of 256 threads: one entry per thread


def _float32_warp_butterfly(per_thread):
    """The xor-shuffle tree over each warp's 32 lanes in float32, then float64 above the warp."""
    v = per_thread.astype(np.float32).reshape(-1, 32).copy()
    for o in (16, 8, 4, 2, 1):
        v = (v + v[:, np.arange(32) ^ o]).astype(np.float32)
    return float(np.sum(v[:, 0].astype(np.float64)))


@pytest.mark.gpu
def test_cancelling_inner_product_is_exact():
    torch, ls = torch_and_lib()
    rng = np.random.default_rng(20)
    lane = np.arange(COUNT) % 32
    frac = rng.integers(0, 8, size=COUNT) / 8.0           # multiples of 1/8, exact next to 2^20 in float32
    b = np.where(lane % 2 == 0, 2.0 ** 20, -(2.0 ** 20)) + frac
    assert np.all(b.astype(np.float32).astype(np.float64) == b)
    exact = float(np.sum(frac))                           # the +-2^20 terms cancel within every warp
    old = _float32_warp_butterfly(b)
    assert abs(old - exact) > 1e-3 * exact                # a float32 warp sum would fail this test
    a_d = torch.ones((1, COUNT), dtype=torch.complex64, device="cuda")
    b_d = torch.from_numpy(b.astype(np.complex64)).reshape(1, COUNT).cuda()
    got = ls.ls_inner_products(a_d, b_d)
    assert got.shape == (1,)
    assert abs(got[0].real - exact) <= 1e-12 * exact and got[0].imag == 0.0


@pytest.mark.gpu
def test_inner_products_of_random_vectors_match_float64():
    torch, ls = torch_and_lib()
    rng = np.random.default_rng(21)
    n = 3 * COUNT + 77   # several entries per thread and a ragged tail
    a = (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).astype(np.complex64)
    b = (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).astype(np.complex64)
    got = ls.ls_inner_products(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    ref = np.sum(np.conj(a.astype(np.complex128)) * b.astype(np.complex128), axis=1)
    scale = np.sqrt(np.sum(np.abs(a) ** 2, axis=1) * np.sum(np.abs(b) ** 2, axis=1))
    assert np.all(np.abs(got - ref) <= 1e-6 * scale)


@pytest.mark.gpu
def test_norm_reduction_keeps_every_lane():
    torch, ls = torch_and_lib()
    lane = np.arange(COUNT) % 32
    pred = np.where(lane == 0, 4096.0, 1.0).astype(np.complex64)   # |d|^2 = 2^24 on lane 0, 1 elsewhere
    exact = (COUNT // 32) * (2.0 ** 24 + 31)
    assert _float32_warp_butterfly(np.abs(pred).astype(np.float64) ** 2) != exact
    p = torch.from_numpy(pred).reshape(1, COUNT).cuda()
    m = torch.zeros_like(p)
    r = torch.empty_like(p)
    loss = ls.ls_residual(p, m, r)
    assert loss[0] == exact
