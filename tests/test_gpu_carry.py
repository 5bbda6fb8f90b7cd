"""Lag-carrying variant of Algorithm 1 on the GPU (PINT_CARRY_LAGS) against
the oracle's (oracle/lagcarry.py): the lagged increments of eqs. (2.4)-(2.5)
carried across the coarse boundaries instead of restarted.

Checks, per coarse time (relative L2 of the coarse coefficient vectors):
the uninterrupted sequential scheme and parareal at a fixed sweep count
match the oracle to 1e-10; k = N reproduces the uninterrupted scheme; the
variant differs from the restarted method.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2411_09244_gb300 import api  # noqa: E402
from paper_2411_09244_gb300.inputs import config_small  # noqa: E402
from oracle import lagcarry as lc  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402


def rel_t(a, b):
    return max(np.linalg.norm(a[n] - b[n]) / np.linalg.norm(b[n]) for n in range(b.shape[0])
               if np.linalg.norm(b[n]) > 0)


@pytest.fixture(scope="module")
def case():
    prob = config_small(n_f=24, nc=4, J=3, ell=2, N=6, P=12, channels=3, contrast=1e4, f_kind="gauss")
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T)
    p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, carry_lags=True)
    yield prob, orc, p
    p.close()


def _oracle_coarse(orc, parts):
    u, w = parts[0], parts[1]
    # the oracle works in the bases' coordinates, like coarse_out
    return np.concatenate([u, w], axis=1)


def test_uninterrupted_sequential_matches_oracle(case):
    prob, orc, p = case
    amp = np.asarray(prob.amp, dtype=np.float64)
    ref = _oracle_coarse(orc, lc.sequential_uninterrupted(orc.sch, orc.u0, orc.w0, orc.F1, orc.F2, amp))
    coarse, fine = p.sequential_solve(prob.u0, prob.f, prob.amp)
    assert rel_t(coarse.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("k", [1, 3])
def test_parareal_after_k_sweeps_matches_oracle(case, k):
    prob, orc, p = case
    amp = np.asarray(prob.amp, dtype=np.float64)
    st = {}
    ref = _oracle_coarse(orc, lc.parareal_carry(orc.sch, orc.u0, orc.w0, orc.F1, orc.F2, amp, eps=0.0, k_max=k,
                                               stats=st))
    coarse, _, s = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=0.0, k_max=k, want_fine=False)
    assert s["K1"] == st["K1"] == k
    assert s["status"] == ("OK" if k == prob.N else "NOT_CONVERGED")
    assert rel_t(coarse.cpu().numpy(), ref) < 1e-10
    # the jump history follows the oracle's
    assert np.allclose(s["jumps"], st["jumps"], rtol=1e-8)


def test_k_equals_N_is_the_uninterrupted_scheme_and_differs_from_restart(case):
    prob, orc, p = case
    cs, _ = p.sequential_solve(prob.u0, prob.f, prob.amp)
    cp, _, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=0.0, k_max=prob.N, want_fine=False)
    assert st["converged"] and st["K1"] == prob.N
    assert rel_t(cp.cpu().numpy(), cs.cpu().numpy()) < 1e-12
    q = api.from_problem(prob, device="cuda", T=orc.T)   # the method: lags restarted
    try:
        cr, _ = q.sequential_solve(prob.u0, prob.f, prob.amp)
    finally:
        q.close()
    assert rel_t(cs.cpu().numpy(), cr.cpu().numpy()) > 1e-8


def test_converges_to_tolerance(case):
    prob, orc, p = case
    cp, _, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=-1e-12, want_fine=False)
    assert st["converged"] and st["K1"] <= prob.N
    cs, _ = p.sequential_solve(prob.u0, prob.f, prob.amp)
    assert rel_t(cp.cpu().numpy(), cs.cpu().numpy()) < 1e-9
