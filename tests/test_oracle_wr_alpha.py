"""The alpha trade-off of the WR fine propagator (Section 4.2, eq. (4.4)), on
the oracle: with the alpha-circulant start the WR error contracts faster for
smaller alpha, while the diagonalisation's round-off grows like 1 / alpha
(the scaling Lambda = diag(alpha^(-p/P)) of eq. (4.6)), so the attainable
accuracy drops.  (Section 5 of the paper words the first half the other way
round; the numbers here follow the alpha-circulant analysis.)"""
import numpy as np
import pytest

from oracle.pipeline import OracleRun
from oracle.scheme import Scheme


@pytest.fixture(scope="module")
def run(small_problem):
    return OracleRun(small_problem)


def _wr(run, alpha):
    prob = run.prob
    sch = Scheme(run.red, run.T, prob.N, prob.P, alpha)
    hist = []
    ends, it = sch.F_wr([(run.u0, run.w0)], [run.F1], [run.F2], wr_tol=1e-13, wr_max=200, history=hist)
    us, _ = sch.F_seq(run.u0, run.w0, run.F1, run.F2)
    return it, np.abs(ends[0][0] - us).max() / np.abs(us).max(), np.array(hist)


def test_smaller_alpha_contracts_faster(run):
    it1, _, h1 = _wr(run, 1e-1)
    it2, _, h2 = _wr(run, 1e-2)
    it4, _, h4 = _wr(run, 1e-4)
    assert it4 < it2 < it1 < 200
    r1 = np.median(h1[3:10] / h1[2:9])
    r4 = np.median(h4[3:8] / h4[2:7])
    assert r4 < r1


def test_round_off_grows_as_alpha_shrinks(run):
    _, e1, _ = _wr(run, 1e-1)
    _, e6, _ = _wr(run, 1e-6)
    assert e1 < 1e-12
    assert e6 > 10 * e1
