"""Pins of the FGP evaluation of prox_{lam TV + i_{>=0}} (Alg. 1, prox step; Beck and Teboulle's FGP)."""
import numpy as np
import pytest

from oracle import tv


def test_grad_and_div_are_negative_adjoints():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((5, 6, 7))
    p = rng.standard_normal((3, 5, 6, 7))
    assert abs(float((tv.grad3(a) * p).sum() + (a * tv.div3(p)).sum())) < 1e-10


def test_gradient_norm_bound_used_for_the_step():
    # ||D||^2 <= 12 in 3-D: the power iteration on D^T D stays below it
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 7, 8))
    for _ in range(300):
        x = -tv.div3(tv.grad3(x))
        x /= np.linalg.norm(x)
    assert float(np.vdot(x, -tv.div3(tv.grad3(x)))) <= 12.0


def test_zero_weight_is_the_projection_on_the_nonnegative_orthant():
    z = np.random.default_rng(0).standard_normal((4, 5, 6))
    assert np.array_equal(tv.prox_tv_nonneg(z, 0.0, 10), np.maximum(z, 0.0))


def test_one_dimensional_case_matches_a_quadratic_program():
    # on an n x 1 x 1 grid TV is sum |x_{i+1} - x_i|: the prox is the QP
    #   min 0.5 ||x - z||^2 + lam sum s_i,  s_i >= +-(x_{i+1} - x_i),  x >= 0
    scipy_opt = pytest.importorskip("scipy.optimize")
    z = np.array([0.3, 1.2, 1.0, -0.4, 0.8, 0.9, 0.1])
    lam, n = 0.25, z.size
    got = tv.prox_tv_nonneg(z.reshape(n, 1, 1), lam, 20000).ravel()

    def obj(w):
        return 0.5 * np.sum((w[:n] - z) ** 2) + lam * np.sum(w[n:])

    cons = []
    for i in range(n - 1):
        cons.append({"type": "ineq", "fun": lambda w, i=i: w[n + i] - (w[i + 1] - w[i])})
        cons.append({"type": "ineq", "fun": lambda w, i=i: w[n + i] + (w[i + 1] - w[i])})
    w0 = np.concatenate([np.maximum(z, 0), np.abs(np.diff(np.maximum(z, 0)))])
    res = scipy_opt.minimize(obj, w0, constraints=cons, bounds=[(0, None)] * n + [(0, None)] * (n - 1),
                             method="SLSQP", options={"ftol": 1e-14, "maxiter": 1000})
    assert res.success
    assert np.max(np.abs(got - res.x[:n])) < 1e-5


def test_three_dimensional_result_is_a_constrained_minimiser():
    rng = np.random.default_rng(0)
    z = rng.standard_normal((6, 7, 8))
    lam = 0.3
    x = tv.prox_tv_nonneg(z, lam, 3000)

    def obj(v):
        return 0.5 * np.sum((v - z) ** 2) + lam * tv.tv(v)

    assert x.min() >= 0.0
    best = obj(x)
    for _ in range(100):
        y = np.maximum(x + 1e-3 * rng.standard_normal(x.shape), 0)
        assert obj(y) >= best - 1e-7
    # the prox does not increase TV and moves towards z's non-negative part
    assert tv.tv(x) <= tv.tv(np.maximum(z, 0))


def test_a_planted_sign_error_in_the_divergence_fails_the_adjoint_pin():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((4, 4, 4))
    p = rng.standard_normal((3, 4, 4, 4))
    bad = -tv.div3(p)
    assert abs(float((tv.grad3(a) * p).sum() + (a * bad).sum())) > 1e-3
