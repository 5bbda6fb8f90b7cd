"""CUDA path vs the FP64 oracle, stage by stage, through the C ABI.

Tolerances: the FP64 path must match the oracle to rel 1e-10 on the coarse
states and fields (the multiscale spaces are canonical, so the reduced
matrices themselves are compared entrywise at 1e-9 relative to their norm).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2411_09244_gb300 import api  # noqa: E402
from paper_2411_09244_gb300.inputs import config_small, config_c1  # noqa: E402
from oracle.pipeline import OracleRun  # noqa: E402


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rel_t(a, b):
    """Largest relative L2 difference over the rows (coarse times) of b that
    do not vanish: an error in a small early state is not hidden by the
    larger later ones."""
    a = np.asarray(a)
    b = np.asarray(b)
    errs = [np.linalg.norm(a[n] - b[n]) / np.linalg.norm(b[n]) for n in range(b.shape[0])
            if np.linalg.norm(b[n]) > 0]
    return max(errs)


CASES = {
    "small16": dict(n_f=16, nc=4, J=2, ell=1, N=4, P=8),
    "ragged24": dict(n_f=24, nc=4, J=3, ell=2, N=3, P=12, channels=3, contrast=1e4, f_kind="gauss"),
    "nlmc_only": dict(n_f=16, nc=4, J=0, ell=1, N=4, P=8, channels=3),
    "uniform": dict(n_f=16, nc=4, J=2, ell=2, N=2, P=16, channels=0, contrast=1.0, u0_kind="sin",
                    f_kind="zero"),
}


@pytest.fixture(scope="module", params=list(CASES) + ["c1"])
def pair(request):
    if request.param == "c1":
        prob = config_c1()
    else:
        prob = config_small(**CASES[request.param])
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T)
    yield request.param, prob, orc, p
    p.close()


def test_dimensions_and_kinds(pair):
    _, prob, orc, p = pair
    assert p.info["d1"] == orc.red.d1 and p.info["d2"] == orc.red.d2
    assert p.info["L"] == orc.spc.L
    kinds = p.get_reduced("kinds").cpu().numpy()
    assert np.array_equal(kinds[:, 0].astype(int), orc.spc.kind)
    assert np.array_equal(kinds[:, 1].astype(int), orc.spc.owner)


@pytest.mark.parametrize("name", ["M11", "A11", "M22", "A22", "M12", "A12"])
def test_reduced_matrices(pair, name):
    _, prob, orc, p = pair
    got = p.get_reduced(name).cpu().numpy()
    ref = getattr(orc.red, name)
    assert rel(got, ref) < 1e-9


def test_gamma_and_lambda(pair):
    _, prob, orc, p = pair
    assert abs(p.info["gamma"] - orc.gamma) < 1e-9
    assert abs(p.info["lambda_max22"] - orc.lam22) < 1e-9 * orc.lam22


def test_load_vector(pair):
    _, prob, orc, p = pair
    got = p.get_reduced("load", prob.f).cpu().numpy()
    ref = np.concatenate([orc.F1, orc.F2])
    assert rel(got, ref) < 1e-10


def test_coarse_and_fine_propagators(pair):
    _, prob, orc, p = pair
    rng = np.random.default_rng(3)
    d1, d2 = orc.red.d1, orc.red.d2
    cnt = min(prob.N, 3)
    X = rng.normal(size=(cnt, d1 + d2))
    amp = prob.amp[:cnt]
    G = p.apply_G(X, prob.f, amp).cpu().numpy()
    for n in range(cnt):
        gu, gw = orc.sch.G(X[n, :d1], X[n, d1:], amp[n] * orc.F1, amp[n] * orc.F2)
        assert rel(G[n], np.concatenate([gu, gw])) < 1e-10
    F, it = p.apply_F(X, prob.f, amp, wr_tol=1e-13, wr_max=400)
    F = F.cpu().numpy()
    starts = [(X[n, :d1], X[n, d1:]) for n in range(cnt)]
    ends, it_o = orc.sch.F_wr(starts, [a * orc.F1 for a in amp], [a * orc.F2 for a in amp], 1e-13, 400)
    assert abs(it - it_o) <= 1
    for n in range(cnt):
        ref = np.concatenate(ends[n])
        assert rel(F[n], ref) < 1e-10
        us, ws = orc.sch.F_seq(X[n, :d1], X[n, d1:], amp[n] * orc.F1, amp[n] * orc.F2)
        assert rel(F[n], np.concatenate([us, ws])) < 1e-9


def test_parareal_solve_matches_oracle(pair):
    _, prob, orc, p = pair
    coarse, fine, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-11, wr_tol=1e-14, wr_max=400)
    u, w, st_o = orc.solve(eps=1e-11, wr_tol=1e-14, wr_max=400)
    ref = np.concatenate([u, w], axis=1)
    assert st["K1"] == st_o["K1"]
    assert rel_t(coarse.cpu().numpy(), ref) < 1e-10
    ref_f = orc.fine_field(u, w)[1:]
    assert rel_t(fine.cpu().numpy(), ref_f) < 1e-10


def test_streaming_coarse_sweep_matches_resident(pair):
    """The FP64 coarse sweep keeps each block's coupling rows in shared
    memory when they fit and reads them from global memory at every step
    otherwise; both variants form the same products and sums, so a solve
    with residency switched off agrees with the default one to rounding noise
    (and so with the oracle)."""
    _, prob, orc, p = pair
    kw = dict(eps=1e-11, wr_tol=1e-14, wr_max=400, want_fine=False)
    c0, _, s0 = p.parareal_solve(prob.u0, prob.f, prob.amp, **kw)
    p.lib.pint_set_sweep_smem(0)
    try:
        c1, _, s1 = p.parareal_solve(prob.u0, prob.f, prob.amp, **kw)
    finally:
        p.lib.pint_set_sweep_smem(-1)
    assert s1["K1"] == s0["K1"]
    assert rel_t(c1.cpu().numpy(), c0.cpu().numpy()) < 1e-14


def test_k_equals_N_matches_sequential(pair):
    _, prob, orc, p = pair
    c_seq, f_seq = p.sequential_solve(prob.u0, prob.f, prob.amp)
    u_s, w_s = orc.sequential()
    assert rel_t(c_seq.cpu().numpy(), np.concatenate([u_s, w_s], axis=1)) < 1e-10
    coarse, _, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=0.0, k_max=prob.N, wr_tol=0.0,
                                     wr_max=400, want_fine=False)
    assert st["K1"] == prob.N
    # k = N reproduces the sequential fine scheme (the bound the oracle meets)
    assert rel_t(coarse.cpu().numpy(), c_seq.cpu().numpy()) < 1e-12


def test_prolongation(pair):
    _, prob, orc, p = pair
    rng = np.random.default_rng(9)
    X = rng.normal(size=(2, orc.red.d1 + orc.red.d2))
    got = p.prolong(X).cpu().numpy()
    ref = np.stack([orc.red.prolong(x[:orc.red.d1], x[orc.red.d1:]) for x in X])
    assert rel(got, ref) < 1e-10


def test_unstable_dt_is_rejected():
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
    p = api.Pint(prob.n_f, prob.kappa)
    p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
    from paper_2411_09244_gb300._lib import PintError
    with pytest.raises(PintError, match="UNSTABLE_DT"):
        p.assemble_reduced(1.0, prob.N, prob.P, prob.alpha)
    info = p.assemble_reduced(1.0, prob.N, prob.P, prob.alpha, allow_unstable=True)
    assert info["dt_max"] < 1.0 / prob.N
    p.close()


def test_bad_arguments_return_codes():
    from paper_2411_09244_gb300._lib import PintError
    k = np.ones((16, 16))
    with pytest.raises(PintError, match="BAD_ARG"):
        api.Pint(3, np.ones((3, 3)))
    k2 = k.copy()
    k2[3, 3] = -1.0
    with pytest.raises(PintError, match="BAD_ARG"):
        api.Pint(16, k2)
    p = api.Pint(16, k)
    with pytest.raises(PintError, match="BAD_ARG"):
        p.build_multiscale_spaces(5, 2, 1)   # 5 does not divide 16
    with pytest.raises(PintError, match="STATE"):
        p.assemble_reduced(1e-3, 4, 8, 0.1)
    p.build_multiscale_spaces(4, 2, 1)
    from paper_2411_09244_gb300._lib import PINT_MIXED
    p.assemble_reduced(None, 4, 8, 0.1)
    nn = 17 * 17
    ref, _, _ = p.parareal_solve(np.zeros(nn), np.ones(nn), eps=1e-10, want_fine=False)
    for bad in (dict(fine_sequential=True), dict(carry_lags=True)):  # FP64 comparison modes only
        with pytest.raises(PintError, match="BAD_ARG"):
            p.assemble_reduced(None, 4, 8, 0.1, precision=PINT_MIXED, **bad)
    # a call refused in its argument checks leaves the assembled time grid in place
    again, _, st = p.parareal_solve(np.zeros(nn), np.ones(nn), eps=1e-10, want_fine=False)
    assert st["status"] == "OK"
    assert float((again - ref).abs().max()) <= 1e-9 * float(ref.abs().max())
    p.close()


@pytest.mark.parametrize("options", ["default", "fp64", "grid", "grid_stream"])
def test_mixed_path_matches_oracle(pair, options):
    """Mixed path (FP32 WR + trajectory refinement) vs the FP64 oracle: max
    over coarse times of the relative L2 error <= 1e-6; "fp64" also runs
    every coarse sweep and the refinement residual in FP64 (PINT_COARSE_FP64
    | PINT_REFINE_FP64); "grid" runs the first solve's FP32 coarse sweeps on
    the grid-wide kernel instead of a cluster (PINT_COARSE_GRID);
    "grid_stream" also streams every grid-wide sweep's coupling rows from
    global memory (pint_set_sweep_smem(0)), the form large couplings take."""
    from paper_2411_09244_gb300._lib import PINT_MIXED, PINT_FP64
    _, prob, orc, p = pair
    p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED, coarse_fp64=options == "fp64",
                       refine_fp64=options == "fp64", coarse_grid=options.startswith("grid"))
    if options == "grid_stream":
        p.lib.pint_set_sweep_smem(0)
    try:
        coarse, fine, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-11, wr_tol=1e-14, wr_max=400)
    finally:
        p.lib.pint_set_sweep_smem(-1)
        p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_FP64)
    u, w = orc.sequential()
    ref = orc.fine_field(u, w)[1:]
    got = fine.cpu().numpy()
    per_t = [rel(got[n], ref[n]) for n in range(prob.N) if np.linalg.norm(ref[n]) > 0]
    assert max(per_t) < 1e-6, max(per_t)


def test_sequential_batched_fine_propagator(pair):
    """PINT_FINE_SEQUENTIAL: Algorithm 1 with F* stepped on all intervals at
    once reaches the same fixed point as the WR fine propagator (and k = N
    reproduces the sequential fine scheme)."""
    name, prob, orc, p = pair
    q = api.Pint(prob.n_f, prob.kappa)
    try:
        q.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
        q.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, fine_sequential=True)
        cs, fs, st = q.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-13, k_max=prob.N)
        cq, fq = q.sequential_solve(prob.u0, prob.f, prob.amp)
    finally:
        q.close()
    assert rel_t(cs.cpu().numpy(), cq.cpu().numpy()) < 1e-10
    u, w = orc.sequential()
    ref = orc.fine_field(u, w)[1:]
    assert rel_t(fs.cpu().numpy(), ref) < 1e-10


def test_paper_example_shape_non_power_of_two_P():
    """The paper's first experiment uses P = 30 fine steps per interval (N = 20): the
    time solve then runs the generic (non power-of-two) DFT kernels on both paths.
    Algorithm 1 must reach the sequential fine scheme: FP64 to 1e-10, mixed to 1e-6."""
    from paper_2411_09244_gb300._lib import PINT_MIXED, PINT_FP64
    prob = config_small(n_f=40, nc=4, J=2, ell=2, N=20, P=30, channels=3, contrast=1e4, f_kind="gauss")
    orc = OracleRun(prob)
    u, w = orc.sequential()
    ref = orc.fine_field(u, w)[1:]
    p = api.from_problem(prob, device="cuda", T=orc.T)
    try:
        _, f64, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-13, wr_tol=1e-15, wr_max=400)
        assert rel_t(f64.cpu().numpy(), ref) < 1e-10
        p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        _, fm, _ = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-13, wr_max=400)
        assert rel_t(fm.cpu().numpy(), ref) < 1e-6
    finally:
        p.close()


def test_mixed_solve_after_reassembly_matches_fresh_context():
    """The WR iterations of the mixed path are replayed from captured CUDA graphs
    that refer to the context's buffers; re-assembling with another time grid
    reallocates them, and the next solve must equal a fresh context's."""
    from paper_2411_09244_gb300._lib import PINT_MIXED
    prob = config_small(n_f=24, nc=4, J=3, ell=2, N=6, P=16, channels=3, contrast=1e4, f_kind="gauss")
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T)
    q = api.from_problem(prob, device="cuda", T=orc.T)
    try:
        p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)          # captures graphs
        p.assemble_reduced(orc.T, 12, 8, prob.alpha, precision=PINT_MIXED)  # other grid (stable: smaller Delta t)
        p.parareal_solve(prob.u0, prob.f, np.ones(12), eps=1e-12)
        p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        _, fp, sp = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)
        q.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        _, fq, sq = q.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)
        assert sp["K1"] == sq["K1"] and sp["wr_total"] == sq["wr_total"]
        assert rel(fp.cpu().numpy(), fq.cpu().numpy()) < 1e-9
    finally:
        p.close()
        q.close()


def test_reassembly_with_new_time_step_and_alpha_matches_fresh_context():
    """The captured WR iterations hold dt and alpha as kernel arguments:
    re-assembling with the same N and P but another T and alpha must not
    replay them (the solve must equal a fresh context's)."""
    from paper_2411_09244_gb300._lib import PINT_MIXED
    prob = config_small(n_f=24, nc=4, J=3, ell=2, N=6, P=16, channels=3, contrast=1e4, f_kind="gauss")
    orc = OracleRun(prob)
    T2, a2 = 0.5 * orc.T, 0.05
    p = api.from_problem(prob, device="cuda", T=orc.T)
    q = api.from_problem(prob, device="cuda", T=T2)
    try:
        p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)          # captures graphs
        p.assemble_reduced(T2, prob.N, prob.P, a2, precision=PINT_MIXED)
        _, fp, sp = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)
        q.assemble_reduced(T2, prob.N, prob.P, a2, precision=PINT_MIXED)
        _, fq, sq = q.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12)
        assert sp["K1"] == sq["K1"] and sp["wr_total"] == sq["wr_total"]
        assert rel_t(fp.cpu().numpy(), fq.cpu().numpy()) < 1e-9
    finally:
        p.close()
        q.close()


def test_library_picks_the_stable_final_time():
    """T <= 0: the library picks 90% of the Section 3.2 bound on the coarse
    step, rounded down to two significant digits, and reports it."""
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
    orc = OracleRun(prob)
    p = api.Pint(prob.n_f, prob.kappa)
    try:
        p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
        info = p.assemble_reduced(None, prob.N, prob.P, prob.alpha)
        assert info["T"] == pytest.approx(orc.T, rel=1e-12)
        assert info["Dt"] == pytest.approx(info["T"] / prob.N, rel=1e-15)
        assert info["Dt"] <= info["dt_max"]
        assert p.T == info["T"]
    finally:
        p.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_bounded_wait_timeout_returns_status_and_context_recovers(mixed):
    """Failure detection without a device fault: with the grid-barrier wait
    limit at zero every wait gives up at once, the coarse sweep records the
    expiry and returns, and the solve returns TIMEOUT (on the mixed path the
    FP64 sweeps of the correction solve, whose flag is read with the jump at
    the end of the iteration); with the limit restored the same context
    solves as before."""
    from paper_2411_09244_gb300._lib import PintError, PINT_MIXED, PINT_FP64
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T, precision=PINT_MIXED if mixed else PINT_FP64)
    try:
        c0, _, s0 = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12, want_fine=False)
        p.lib.pint_set_wait_limit(0)
        try:
            with pytest.raises(PintError, match="TIMEOUT"):
                p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12, want_fine=False)
        finally:
            p.lib.pint_set_wait_limit(-1)
        c1, _, s1 = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-12, want_fine=False)
        assert s1["converged"] == s0["converged"] and s1["K1"] == s0["K1"]
        # FP64: the same arithmetic; mixed: FP32 atomics in the WR norms may
        # reorder, so the same answer to well inside the mixed tolerance
        assert rel_t(c1.cpu().numpy(), c0.cpu().numpy()) < (1e-9 if mixed else 1e-14)
    finally:
        p.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_not_converged_and_nonfinite_statuses(mixed):
    """Failure statuses without any device fault: k_max below what eps needs
    returns NOT_CONVERGED with the outputs and the jump history written; a
    non-finite source makes the WR update norm non-finite and the solve
    returns NONFINITE."""
    from paper_2411_09244_gb300._lib import PINT_MIXED, PintError
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=6, P=8, f_kind="gauss")
    orc = OracleRun(prob)
    p = api.from_problem(prob, device="cuda", T=orc.T)
    try:
        if mixed:
            p.assemble_reduced(orc.T, prob.N, prob.P, prob.alpha, precision=PINT_MIXED)
        coarse, fine, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-300, k_max=1)
        assert st["status"] == "NOT_CONVERGED" and not st["converged"]
        assert st["jumps"][0] > 0 and np.isfinite(coarse.cpu().numpy()).all()
        assert np.isfinite(fine.cpu().numpy()).all()
        bad = np.array(prob.f, dtype=np.float64)
        bad[len(bad) // 2] = np.nan
        with pytest.raises(PintError, match="NONFINITE"):
            p.parareal_solve(prob.u0, bad, prob.amp, eps=1e-10)
        # the context stays usable
        _, _, st2 = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-10)
        assert st2["converged"]
    finally:
        p.close()


def test_wr_alpha_trade_off_on_the_gpu():
    """The FP64 WR fine propagator on the GPU shows the oracle's alpha trade-off
    (tests/test_oracle_wr_alpha.py): fewer iterations for alpha = 1e-4 than
    1e-1, and a round-off floor far above the 1e-1 error at alpha = 1e-6."""
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
    orc = OracleRun(prob)
    x = np.concatenate([orc.u0, orc.w0])[None, :]
    us, ws = orc.sch.F_seq(orc.u0, orc.w0, orc.F1, orc.F2)
    ref = np.concatenate([us, ws])
    p = api.from_problem(prob, device="cuda", T=orc.T)
    res = {}
    try:
        for alpha in (1e-1, 1e-4, 1e-6):
            p.assemble_reduced(orc.T, prob.N, prob.P, alpha)
            F, it = p.apply_F(x, prob.f, np.ones(1), wr_tol=1e-13, wr_max=200)
            res[alpha] = (it, rel(F.cpu().numpy()[0], ref))
    finally:
        p.close()
    assert res[1e-4][0] < res[1e-1][0] < 200
    assert res[1e-1][1] < 1e-11
    assert res[1e-6][1] > 10 * res[1e-1][1]
