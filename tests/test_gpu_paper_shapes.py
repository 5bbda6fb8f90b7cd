"""The paper's experiment shapes (Section 5) as seeded stand-ins (its fields
are figure images only): the grid h = 1/100, H = 1/10 with N = 20 intervals
of P = 30 fine steps (non-power-of-two P: the time solve's DFTs run as
products with the DFT matrix), the sweep over N at fixed N P = 600, and a
sweep over the final time at a fixed coarse step.

Parity: per coarse time against the oracle's sequential fine scheme, FP64
path <= 1e-10, mixed path <= 1e-6.  The sweeps check the paper's qualitative
claims: parareal iterations stay stable as N grows at fixed N P, and the
method converges at every final time of the sweep.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2411_09244_gb300 import api, _lib  # noqa: E402
from paper_2411_09244_gb300.inputs import config_paper_grid  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402


def per_time_rel(got, ref):
    return np.array([np.linalg.norm(got[n] - ref[n]) / np.linalg.norm(ref[n]) for n in range(ref.shape[0])
                     if np.linalg.norm(ref[n]) > 0])


@pytest.fixture(scope="module")
def paper_grid():
    prob = config_paper_grid(N=20, P=30)
    orc = OracleRun(prob)
    u, w = orc.sequential()
    ref = orc.fine_field(u, w)[1:]
    p = api.from_problem(prob, device="cuda", T=orc.T)
    yield prob, orc, ref, p
    p.close()


def test_paper_grid_dimensions(paper_grid):
    prob, orc, ref, p = paper_grid
    assert (prob.n_f, prob.nc) == (100, 10)
    assert (p.info["d1"], p.info["d2"]) == (orc.red.d1, orc.red.d2)
    assert abs(p.info["gamma"] - orc.gamma) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_grid_p30_matches_oracle(paper_grid, precision):
    prob, orc, ref, p = paper_grid
    prec = _lib.PINT_FP64 if precision == "fp64" else _lib.PINT_MIXED
    p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=prec)
    eps, tol = (-1e-13, 1e-10) if precision == "fp64" else (-1e-12, 1e-6)
    _, fine, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=eps, wr_tol=-1e-16 if precision == "fp64" else None,
                                   wr_max=400)
    assert st["converged"]
    err = per_time_rel(fine.cpu().numpy(), ref)
    assert err.size == prob.N and err.max() <= tol, (precision, err.max(), st["K1"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_iterations_stable_in_N_at_fixed_NP(precision):
    """N P = 600 (the paper's first experiment): N = 20, 30, 40, 60 intervals of
    P = 30, 20, 15, 10 steps on one final time (the stable T of N = 20); the
    parareal sweeps to a relative jump tolerance of 1e-10 grow far slower
    than N: tripling N adds less than half (measured 16, 18, 20, 22)."""
    prob0 = config_paper_grid(N=20, P=30)
    p = api.Pint(prob0.n_f, prob0.kappa)
    prec = _lib.PINT_FP64 if precision == "fp64" else _lib.PINT_MIXED
    K = {}
    try:
        p.build_multiscale_spaces(prob0.nc, prob0.J, prob0.ell)
        T = p.assemble_reduced(None, 20, 30, prob0.alpha)["T"]      # stable for the coarsest N
        for N in (20, 30, 40, 60):
            P = 600 // N
            prob = config_paper_grid(N=N, P=P)
            p.assemble_reduced(T, N, P, prob.alpha, precision=prec)
            _, _, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=-1e-10, want_fine=False)
            assert st["converged"], (N, st)
            K[N] = st["K1"]
    finally:
        p.close()
    assert K[60] <= 1.5 * K[20] and all(K[a] <= K[b] + 1 for a, b in ((20, 30), (30, 40), (40, 60))), K


def test_final_time_sweep_at_fixed_coarse_step():
    """Fixed Delta t and dt (P = 20), final times T0, 1.5 T0, 2 T0 with N = 10,
    15, 20 (the shape of the paper's T-sweeps): every solve converges and
    matches the sequential fine scheme of its own grid."""
    prob0 = config_paper_grid(N=10, P=20)
    p = api.Pint(prob0.n_f, prob0.kappa)
    try:
        p.build_multiscale_spaces(prob0.nc, prob0.J, prob0.ell)
        T0 = p.assemble_reduced(None, 10, 20, prob0.alpha)["T"]
        for N, T in ((10, T0), (15, 1.5 * T0), (20, 2.0 * T0)):
            prob = config_paper_grid(N=N, P=20)
            p.assemble_reduced(T, N, 20, prob.alpha)
            assert p.info["Dt"] == pytest.approx(T0 / 10, rel=1e-12)
            _, fine, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=-1e-13, wr_tol=-1e-16, wr_max=400)
            _, seq = p.sequential_solve(prob.u0, prob.f, prob.amp)
            assert st["converged"] and st["K1"] <= N
            assert per_time_rel(fine.cpu().numpy(), seq.cpu().numpy()).max() < 1e-10
    finally:
        p.close()
