"""Pins of the oracle's lag-carrying variant of Algorithm 1 (lagged increments
carried across coarse boundaries instead of restarted).

The uninterrupted fine scheme is checked against the same scheme run as one
interval of N P steps (its only restart is at t = 0), parareal at k = N against
the uninterrupted scheme, and P = 1 (where the coarse and fine steps coincide
and the interpolated lag is exact) against one-sweep convergence.
"""
import numpy as np
import pytest

from oracle import lagcarry as lc
from oracle import parareal as pr
from oracle.pipeline import OracleRun
from oracle.scheme import Scheme


@pytest.fixture(scope="module")
def run(small_problem):
    return OracleRun(small_problem)


def test_uninterrupted_equals_one_long_interval(run):
    sch, prob = run.sch, run.prob
    amp = np.ones(prob.N)
    u, w, ul, wl = lc.sequential_uninterrupted(sch, run.u0, run.w0, run.F1, run.F2, amp)
    one = Scheme(run.red, sch.T, 1, prob.N * prob.P, prob.alpha)   # restart only at t = 0
    u1, w1 = pr.sequential_fine(one, run.u0, run.w0, run.F1, run.F2, np.ones(1))
    scale = np.abs(u1).max()
    assert np.abs(u[-1] - u1[-1]).max() < 1e-12 * scale
    assert np.abs(w[-1] - w1[-1]).max() < 1e-12 * max(np.abs(w1).max(), 1e-300)


def test_carry_differs_from_restart(run):
    # the variant is not the method: carrying the lags changes the solution
    sch, prob = run.sch, run.prob
    amp = np.asarray(prob.amp, dtype=np.float64)
    uc, wc, _, _ = lc.sequential_uninterrupted(sch, run.u0, run.w0, run.F1, run.F2, amp)
    ur, wr = pr.sequential_fine(sch, run.u0, run.w0, run.F1, run.F2, amp)
    d = np.abs(uc[-1] - ur[-1]).max() / np.abs(ur[-1]).max()
    assert d > 1e-8


def test_parareal_k_equals_N_is_the_uninterrupted_scheme(run):
    sch, prob = run.sch, run.prob
    amp = np.asarray(prob.amp, dtype=np.float64)
    ref = lc.sequential_uninterrupted(sch, run.u0, run.w0, run.F1, run.F2, amp)
    st = {}
    got = lc.parareal_carry(sch, run.u0, run.w0, run.F1, run.F2, amp, eps=0.0, k_max=prob.N, stats=st)
    assert st["K1"] == prob.N
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() < 1e-12 * max(np.abs(b).max(), 1e-300)
    # states n <= k are exact after k sweeps
    got2 = lc.parareal_carry(sch, run.u0, run.w0, run.F1, run.F2, amp, eps=0.0, k_max=2)
    assert np.abs(got2[0][:3] - ref[0][:3]).max() < 1e-12 * np.abs(ref[0]).max()


def test_jumps_contract(run):
    sch, prob = run.sch, run.prob
    amp = np.asarray(prob.amp, dtype=np.float64)
    st = {}
    lc.parareal_carry(sch, run.u0, run.w0, run.F1, run.F2, amp, eps=1e-14, k_max=prob.N, stats=st)
    j = np.array(st["jumps"])
    assert len(j) >= 2 and np.all(j[1:] < j[:-1])


def test_single_fine_step_per_interval_converges_in_one_sweep(run):
    # P = 1: the coarse step is the fine step and the interpolated lag is the
    # exact previous state, so G = F and the first sweep changes nothing
    prob = run.prob
    sch1 = Scheme(run.red, run.sch.T, prob.N, 1, prob.alpha)
    amp = np.asarray(prob.amp, dtype=np.float64)
    st = {}
    got = lc.parareal_carry(sch1, run.u0, run.w0, run.F1, run.F2, amp, eps=0.0, k_max=2, stats=st)
    ref = lc.sequential_uninterrupted(sch1, run.u0, run.w0, run.F1, run.F2, amp)
    scale = np.abs(ref[0]).max()
    assert st["jumps"][0] < 1e-12 * scale
    assert np.abs(got[0] - ref[0]).max() < 1e-12 * scale
