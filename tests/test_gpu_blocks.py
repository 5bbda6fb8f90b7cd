"""Large coarse blocks (more than 400 nodes: 24- and 32-cell blocks): the
auxiliary eigenproblems of eq. (3.1) run by shift-invert subspace iteration
with a banded Cholesky instead of the dense Jacobi.  Against the oracle
(dense LAPACK per block): the selected functions (kinds, dimensions,
including the cluster completion of degenerate pairs on a uniform block),
gamma, lambda_max(A22, M22), the reduced matrices and the solution per
coarse time (FP64, 1e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2411_09244_gb300 import api  # noqa: E402
from paper_2411_09244_gb300.inputs import config_small  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402

CASES = {
    "blocks32_channels": dict(n_f=64, nc=2, J=3, ell=1, N=4, P=8, channels=3, contrast=1e4, f_kind="gauss"),
    "blocks24_channels": dict(n_f=48, nc=2, J=4, ell=1, N=4, P=8, channels=2, contrast=1e3, f_kind="gauss"),
    "blocks32_uniform": dict(n_f=64, nc=2, J=4, ell=1, N=3, P=8, channels=0, contrast=1.0, u0_kind="sin",
                             f_kind="zero"),
}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_large_blocks_match_oracle(name):
    prob = config_small(**CASES[name])
    assert (prob.n_f // prob.nc + 1) ** 2 > 400
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T)
    try:
        assert (p.info["d1"], p.info["d2"], p.info["L"]) == (orc.red.d1, orc.red.d2, orc.spc.L)
        kinds = p.get_reduced("kinds").cpu().numpy()
        assert np.array_equal(kinds[:, 0].astype(int), orc.spc.kind)
        assert abs(p.info["gamma"] - orc.gamma) < 1e-9
        assert abs(p.info["lambda_max22"] - orc.lam22) < 1e-9 * orc.lam22
        for m in ("M11", "A11", "M22", "A22", "M12", "A12"):
            assert rel(p.get_reduced(m).cpu().numpy(), getattr(orc.red, m)) < 1e-9, m
        u, w = orc.sequential()
        ref = orc.fine_field(u, w)[1:]
        _, fine = p.sequential_solve(prob.u0, prob.f, prob.amp)
        got = fine.cpu().numpy()
        err = max(np.linalg.norm(got[n] - ref[n]) / np.linalg.norm(ref[n]) for n in range(prob.N)
                  if np.linalg.norm(ref[n]) > 0)
        assert err < 1e-10, err
    finally:
        p.close()
