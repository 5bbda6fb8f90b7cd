"""Adjoint (backward) parareal through the C ABI (pint_adjoint) against the
oracle's FP64 adjoint and against central differences of the GPU's own
forward map.  The misfit is quadratic in (u0, amp), so a central difference
with step 1 is exact up to the forward solve's tolerance.

Tolerances: FP64 path vs oracle rel 1e-8; central differences rel 1e-5;
low-precision path (FP32 transposed sweeps, mixed forward) vs oracle rel 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2411_09244_gb300 import api, _lib  # noqa: E402
from paper_2411_09244_gb300.inputs import config_small, config_c3, observation_nodes  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402
from oracle.adjoint import Adjoint  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def small_case(seed=11, N=4, P=8, n_obs=8):
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=N, P=P, seed=seed)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((prob.n_f + 1) ** 2)
    prob.u0 = u0 * (np.arange(u0.size) % 3 != 0)
    prob.amp = 0.5 + rng.random(prob.N)
    obs = observation_nodes(prob.n_f, n_obs, seed=3)
    data = rng.standard_normal((prob.N, obs.size))
    return prob, obs, data


@pytest.fixture(scope="module")
def small():
    prob, obs, data = small_case()
    run = OracleRun(prob)
    adj = Adjoint(run, obs)
    ref = adj.gradient(prob.u0, prob.amp, data)
    return prob, obs, data, run, ref


def test_fp64_adjoint_matches_oracle(small):
    prob, obs, data, run, (J0, gu0, ga0) = small
    p = api.from_problem(prob, T=run.T)
    try:
        J, gu, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-13)
    finally:
        p.close()
    assert J == pytest.approx(J0, rel=1e-10)
    assert rel(gu.cpu().numpy(), gu0) < 1e-8
    assert rel(ga.cpu().numpy(), ga0) < 1e-8


def test_fp64_adjoint_central_differences(small):
    prob, obs, data, run, _ = small
    p = api.from_problem(prob, T=run.T)
    try:
        J, gu, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-13)
        gu, ga = gu.cpu().numpy(), ga.cpu().numpy()

        def misfit(u0, amp):
            _, fine = p.sequential_solve(u0, prob.f, amp)
            y = fine.cpu().numpy()[:, obs]
            return 0.5 * float(np.sum((y - data) ** 2))

        assert misfit(prob.u0, prob.amp) == pytest.approx(J, rel=1e-10)
        rng = np.random.default_rng(9)
        for _ in range(3):
            v = rng.standard_normal(prob.u0.size)
            fd = 0.5 * (misfit(prob.u0 + v, prob.amp) - misfit(prob.u0 - v, prob.amp))
            assert fd == pytest.approx(gu @ v, rel=1e-5)
            q = rng.standard_normal(prob.N)
            fd = 0.5 * (misfit(prob.u0, prob.amp + q) - misfit(prob.u0, prob.amp - q))
            assert fd == pytest.approx(ga @ q, rel=1e-5)
    finally:
        p.close()


def test_low_precision_adjoint_matches_oracle(small):
    prob, obs, data, run, (J0, gu0, ga0) = small
    p = api.from_problem(prob, T=run.T, precision=_lib.PINT_MIXED)
    try:
        J, gu, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-12)
    finally:
        p.close()
    assert J == pytest.approx(J0, rel=1e-5)
    assert rel(gu.cpu().numpy(), gu0) < 1e-4
    assert rel(ga.cpu().numpy(), ga0) < 1e-4


def test_autograd_function(small):
    prob, obs, data, run, (J0, gu0, ga0) = small
    p = api.from_problem(prob, T=run.T)
    try:
        u0 = torch.tensor(prob.u0, dtype=torch.float64, device="cuda", requires_grad=True)
        amp = torch.tensor(prob.amp, dtype=torch.float64, device="cuda", requires_grad=True)
        J = api.ObservationMisfit.apply(u0, amp, p, obs, data, prob.f, {"eps": 1e-13})
        (2.0 * J).backward()
    finally:
        p.close()
    assert float(J.detach()) == pytest.approx(J0, rel=1e-10)
    assert rel(u0.grad.cpu().numpy(), 2.0 * gu0) < 1e-8
    assert rel(amp.grad.cpu().numpy(), 2.0 * ga0) < 1e-8


def test_adjoint_bad_args(small):
    prob, obs, data, run, _ = small
    p = api.from_problem(prob, T=run.T)
    try:
        bad = np.array([0, (prob.n_f + 1) ** 2], dtype=np.int32)
        with pytest.raises(_lib.PintError):
            p.adjoint(bad, data[:, :2], prob.u0, prob.f, prob.amp)
    finally:
        p.close()


@pytest.mark.slow
def test_c3_fp64_central_differences():
    """128x128 / 16x16 / J=3 / N=32 x P=32 workload: FP64 gradient against
    central differences of the GPU forward (parareal to a tight tolerance)."""
    prob = config_c3()
    obs = observation_nodes(prob.n_f, 64, seed=prob.n_f)
    rng = np.random.default_rng(21)
    data = rng.standard_normal((prob.N, obs.size))
    p = api.from_problem(prob)
    try:
        J, gu, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-12)
        gu, ga = gu.cpu().numpy(), ga.cpu().numpy()

        def misfit(u0, amp):
            Jv, _, _ = p.adjoint(obs, data, u0, prob.f, amp, eps=1e-12)
            return Jv

        for _ in range(2):
            v = rng.standard_normal(prob.u0.size)
            fd = 0.5 * (misfit(prob.u0 + v, prob.amp) - misfit(prob.u0 - v, prob.amp))
            assert fd == pytest.approx(gu @ v, rel=1e-5)
            q = rng.standard_normal(prob.N)
            fd = 0.5 * (misfit(prob.u0, prob.amp + q) - misfit(prob.u0, prob.amp - q))
            assert fd == pytest.approx(ga @ q, rel=1e-5)
    finally:
        p.close()


def test_amplitude_gradient_routes_agree(small):
    """dJ/da_n by recomputing the fine adjoint inside each interval from the
    boundary adjoint (default) equals the unit-response shortcut
    <lambda_{n+1}, s> (PINT_ADJOINT_RESPONSE) and the oracle's recomputed one."""
    prob, obs, data, run, _ = small
    adj = Adjoint(run, obs)
    _, _, ga_rec = adj.gradient(prob.u0, prob.amp, data, amp_mode="recompute")
    p = api.from_problem(prob, T=run.T)
    try:
        _, _, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-13)
        p.assemble_reduced(run.T, prob.N, prob.P, prob.alpha, adjoint_response=True)
        _, _, ga_s = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-13)
    finally:
        p.close()
    assert rel(ga.cpu().numpy(), ga_s.cpu().numpy()) < 1e-11
    assert rel(ga.cpu().numpy(), ga_rec) < 1e-8


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c3_adjoint_matches_oracle_adjoint(precision):
    """128x128 / 16x16 / J=3 / N=32 x P=32 workload (16 amplitudes held over two
    intervals each, 64 observation nodes): the GPU gradient against the
    oracle's FP64 adjoint with the fine adjoint recomputed inside each
    interval; FP64 path 1e-8, low-precision path 1e-4."""
    prob = config_c3()
    obs = observation_nodes(prob.n_f, 64, seed=prob.n_f)
    rng = np.random.default_rng(21)
    data = rng.standard_normal((prob.N, obs.size))
    run = OracleRun(prob)
    J0, gu0, ga0 = Adjoint(run, obs).gradient(prob.u0, prob.amp, data, amp_mode="recompute")
    prec = _lib.PINT_FP64 if precision == "fp64" else _lib.PINT_MIXED
    p = api.from_problem(prob, T=run.T, precision=prec)
    try:
        J, gu, ga = p.adjoint(obs, data, prob.u0, prob.f, prob.amp, eps=1e-12)
    finally:
        p.close()
    tol = 1e-8 if precision == "fp64" else 1e-4
    assert J == pytest.approx(J0, rel=tol)
    assert rel(gu.cpu().numpy(), gu0) < tol
    assert rel(ga.cpu().numpy(), ga0) < tol
    # the gradient of each of the 16 shared amplitudes sums its two intervals
    g16 = ga.cpu().numpy().reshape(16, 2).sum(axis=1)
    assert rel(g16, ga0.reshape(16, 2).sum(axis=1)) < tol
