"""Pins of the oracle adjoint (oracle/adjoint.py) against what the mathematics
fixes: the misfit is quadratic in (u0, amp), so a central difference with any
step is exact up to rounding; the transpose passes the dot-product identity;
the two routes to the amplitude gradient agree; the dense step matrix
composes to the fine scheme itself."""
import numpy as np
import pytest

from paper_2411_09244_gb300.inputs import config_small, observation_nodes
from oracle.pipeline import OracleRun
from oracle.adjoint import Adjoint


@pytest.fixture(scope="module")
def adj():
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8, seed=11)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((prob.n_f + 1) ** 2)
    prob.u0 = u0 * (np.arange(u0.size) % 3 != 0)
    run = OracleRun(prob)
    obs = observation_nodes(prob.n_f, 8, seed=3)
    a = Adjoint(run, obs)
    data = rng.standard_normal((prob.N, obs.size))
    return a, prob, data


def test_interval_map_is_the_fine_scheme(adj):
    a, prob, _ = adj
    r = a.run
    rng = np.random.default_rng(1)
    x = rng.standard_normal(a.d)
    u, w = r.sch.F_seq(x[:a.d1], x[a.d1:], 0.7 * r.F1, 0.7 * r.F2)
    got = a.Phi(x) + 0.7 * a.unit_response()
    ref = np.concatenate([u, w])
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_transpose_dot_product(adj):
    a, _, _ = adj
    rng = np.random.default_rng(2)
    for _ in range(3):
        x, y = rng.standard_normal(a.d), rng.standard_normal(a.d)
        lhs, rhs = a.Phi(x) @ y, x @ a.Phi_T(y)
        assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(a.Phi(x)) * np.linalg.norm(y))


def test_gradient_matches_central_differences(adj):
    """J quadratic: (J(p + v) - J(p - v)) / 2 = grad . v exactly (step 1)."""
    a, prob, data = adj
    J, gu, ga = a.gradient(prob.u0, prob.amp, data)
    assert J == pytest.approx(a.misfit(prob.u0, prob.amp, data), rel=1e-14)
    rng = np.random.default_rng(3)
    for _ in range(4):
        v = rng.standard_normal(prob.u0.size)
        fd = 0.5 * (a.misfit(prob.u0 + v, prob.amp, data) - a.misfit(prob.u0 - v, prob.amp, data))
        assert fd == pytest.approx(gu @ v, rel=1e-9)
        q = rng.standard_normal(prob.N)
        fd = 0.5 * (a.misfit(prob.u0, prob.amp + q, data) - a.misfit(prob.u0, prob.amp - q, data))
        assert fd == pytest.approx(ga @ q, rel=1e-9)


def test_amplitude_gradient_two_routes(adj):
    a, prob, data = adj
    _, _, g1 = a.gradient(prob.u0, prob.amp, data, amp_mode="response")
    _, _, g2 = a.gradient(prob.u0, prob.amp, data, amp_mode="recompute")
    assert np.linalg.norm(g1 - g2) <= 1e-12 * np.linalg.norm(g1)


def test_zero_residual_zero_gradient(adj):
    """Data equal to the model's own observations: J = 0 and the gradient vanishes."""
    a, prob, _ = adj
    d0 = a.observe(a.forward(prob.u0, prob.amp))
    J, gu, ga = a.gradient(prob.u0, prob.amp, d0)
    assert J == 0.0 or J < 1e-28
    assert np.abs(gu).max() < 1e-12 and np.abs(ga).max() < 1e-12
