"""Pins of the Hessian Schatten-norm prox (Sec. 4.2 regulariser, FGP on the dual)."""
import numpy as np
import pytest

from oracle import hessian as hs


def test_adjoint_in_the_frobenius_inner_product():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 6, 7))
    w = rng.standard_normal((6, 5, 6, 7))
    assert abs(hs.field_dot(hs.hessian(x), w) - float((x * hs.hessian_adjoint(w)).sum())) < 1e-9


def test_hessian_of_a_quadratic_is_its_constant_second_derivative_matrix():
    # interior voxels, unit spacing: second differences of a quadratic are exact
    z, y, x = np.meshgrid(np.arange(7.0), np.arange(8.0), np.arange(9.0), indexing="ij")
    f = 0.5 * 3.0 * z * z - 0.5 * 2.0 * y * y + 0.5 * 5.0 * x * x + 1.5 * z * y - 0.25 * z * x + 0.75 * y * x
    h = hs.hessian(f)
    inner = (slice(1, -1),) * 3
    want = {"zz": 3.0, "yy": -2.0, "xx": 5.0, "zy": 1.5, "zx": -0.25, "yx": 0.75}
    for k, name in enumerate(hs.COMPONENTS):
        assert np.allclose(h[k][inner], want[name], atol=1e-12)


def test_hessian_norm_bound_used_for_the_step():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 7, 8))
    for _ in range(300):
        x = hs.hessian_adjoint(hs.hessian(x))
        x /= np.linalg.norm(x)
    assert float((x * hs.hessian_adjoint(hs.hessian(x))).sum()) <= 144.0


def test_spectral_ball_projection():
    rng = np.random.default_rng(3)
    w = 3.0 * rng.standard_normal((6, 3, 4, 5))
    p = hs.project_spectral_ball(w)
    assert np.max(np.abs(np.linalg.eigvalsh(hs.to_matrices(p)))) <= 1.0 + 1e-12
    assert np.allclose(hs.project_spectral_ball(p), p, atol=1e-12)          # idempotent
    small = 0.1 * w / np.max(np.abs(w))
    assert np.allclose(hs.project_spectral_ball(small), small, atol=1e-12)  # inside: unchanged
    d = np.zeros((6, 1, 1, 1))
    d[:3, 0, 0, 0] = [2.5, -0.3, -4.0]                                      # diagonal: clipped
    assert np.allclose(hs.project_spectral_ball(d)[:, 0, 0, 0], [1.0, -0.3, -1.0, 0, 0, 0], atol=1e-12)
    q = hs.project_spectral_ball(w + 0.5)
    assert hs.field_dot(p - q, p - q) <= hs.field_dot(w - (w + 0.5), w - (w + 0.5)) + 1e-9   # non-expansive


def test_zero_weight_is_the_projection_on_the_nonnegative_orthant():
    z = np.random.default_rng(0).standard_normal((4, 5, 6))
    assert np.array_equal(hs.prox_hs_nonneg(z, 0.0, 10), np.maximum(z, 0.0))


def test_one_dimensional_case_matches_a_quadratic_program():
    # on an n x 1 x 1 grid only D_zz remains: the prox is the QP
    #   min 0.5 ||x - z||^2 + lam sum s_i,  s_i >= +-(D_zz x)_i,  x >= 0
    scipy_opt = pytest.importorskip("scipy.optimize")
    z = np.array([0.3, 1.2, 1.0, -0.4, 0.8, 0.9, 0.1, 0.5])
    lam, n = 0.05, z.size
    got = hs.prox_hs_nonneg(z.reshape(n, 1, 1), lam, 40000).ravel()
    D = -np.diag(np.r_[1.0, 2.0 * np.ones(n - 2), 1.0]) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    assert np.allclose(D @ z, hs.hessian(z.reshape(n, 1, 1))[0].ravel())

    def obj(w):
        return 0.5 * np.sum((w[:n] - z) ** 2) + lam * np.sum(w[n:])

    cons = []
    for i in range(n):
        cons.append({"type": "ineq", "fun": lambda w, i=i: w[n + i] - D[i] @ w[:n]})
        cons.append({"type": "ineq", "fun": lambda w, i=i: w[n + i] + D[i] @ w[:n]})
    x0 = np.maximum(z, 0)
    res = scipy_opt.minimize(obj, np.concatenate([x0, np.abs(D @ x0)]), constraints=cons,
                             bounds=[(0, None)] * (2 * n), method="SLSQP", options={"ftol": 1e-15, "maxiter": 2000})
    assert res.success
    assert np.max(np.abs(got - res.x[:n])) < 1e-4


def test_three_dimensional_result_is_a_constrained_minimiser():
    rng = np.random.default_rng(0)
    z = 0.5 + rng.standard_normal((5, 6, 7))
    lam = 0.05
    x = hs.prox_hs_nonneg(z, lam, 4000)

    def obj(v):
        return 0.5 * np.sum((v - z) ** 2) + lam * hs.hs1(v)

    assert x.min() >= 0.0
    best = obj(x)
    for _ in range(60):
        y = np.maximum(x + 1e-3 * rng.standard_normal(x.shape), 0)
        assert obj(y) >= best - 1e-6
