"""Independent pins of the oracle's scalar diagnostics, initial projection,
closed-form accuracy and constraint weighting.

Each check computes the quantity by a route that shares nothing with the
oracle function under test (fine-grid vectors, Cholesky of the fine mass
matrix, SVD, closed forms, dense KKT solves), so that a plausible mistake in
the oracle (a missing square root, the wrong pencil, the smallest instead of
the largest eigenvalue, a transposed coupling, a dropped block of the Gram
matrix) fails one of them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fem import FineProblem
from oracle.pipeline import OracleRun
from oracle.scheme import Scheme
from oracle.spaces import Window, cem_window
from paper_2411_09244_gb300.inputs import config_small


@pytest.fixture(scope="module")
def run24():
    prob = config_small(n_f=24, nc=4, J=3, ell=2, N=3, P=12, channels=3, contrast=1e4, f_kind="gauss")
    return OracleRun(prob)


def _mass_orthonormal(L, Psi):
    """Orthonormal basis (Euclidean) of L^T Psi: the image of span(Psi) under
    the map v -> L^T v, for which (v, v')_{M_f} = (L^T v) . (L^T v')."""
    Q, _ = np.linalg.qr(L.T @ Psi)
    return Q


def test_gamma_is_cosine_of_smallest_principal_angle(run24):
    """eq. (4.15): gamma = sup over u in V_H1, w in V_H2 of (u, w) / (||u|| ||w||)
    in L2.  Computed here from fine-grid vectors: Cholesky M_f = L L^T, QR of
    L^T Psi1 and L^T Psi2, and the largest singular value of Q1^T Q2 (the
    cosine of the smallest principal angle; Bjorck and Golub 1973)."""
    fp, spc = run24.fp, run24.spc
    L = np.linalg.cholesky(fp.M.toarray())
    Q1 = _mass_orthonormal(L, spc.Psi1)
    Q2 = _mass_orthonormal(L, spc.Psi2)
    cos = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    assert run24.red.gamma() == pytest.approx(cos[0], rel=1e-10)
    # the same angle from scipy's routine (sine-based for small angles)
    ang = sla.subspace_angles(L.T @ spc.Psi1, L.T @ spc.Psi2)
    assert run24.red.gamma() == pytest.approx(np.cos(ang.min()), rel=1e-8)
    # realised by a pair of functions: the cosine of u* = Psi1 a, w* = Psi2 b
    U, s, Vt = np.linalg.svd(Q1.T @ Q2)
    u = Q1 @ U[:, 0]
    w = Q2 @ Vt[0]
    assert abs(u @ w) == pytest.approx(run24.red.gamma(), rel=1e-10)


def test_lambda_max_22_is_the_largest_rayleigh_quotient(run24):
    """Section 3.2: sup over v in V_H2 of ||v||_a^2 / ||v||^2.  Computed from
    fine-grid vectors: an L2-orthonormal basis Q of V_H2 (through L^T) and the
    largest eigenvalue of the symmetric matrix Q^T L^-1 A_f L^-T Q."""
    fp, spc = run24.fp, run24.spc
    A = fp.A.toarray()
    L = np.linalg.cholesky(fp.M.toarray())
    Q = _mass_orthonormal(L, spc.Psi2)
    Linv_A_LinvT = sla.solve_triangular(L, sla.solve_triangular(L, A, lower=True).T, lower=True).T
    H = Q.T @ Linv_A_LinvT @ Q
    lam, vec = np.linalg.eigh(0.5 * (H + H.T))
    got = run24.red.lambda_max_22()
    assert got == pytest.approx(lam[-1], rel=1e-9)
    assert got > 1.5 * lam[0]                       # not the smallest one
    # Rayleigh quotient of the maximiser, as a fine-grid function v = L^-T Q y
    v = sla.solve_triangular(L.T, Q @ vec[:, -1], lower=False)
    rq = (v @ A @ v) / (v @ fp.M @ v)
    assert rq == pytest.approx(got, rel=1e-9)
    # no function of V_H2 exceeds it
    rng = np.random.default_rng(17)
    for _ in range(50):
        x = spc.Psi2 @ rng.normal(size=spc.Psi2.shape[1])
        assert (x @ A @ x) / (x @ fp.M @ x) <= got * (1 + 1e-12)


def test_initial_projection_recovers_functions_of_v_h(run24):
    """eq. (2.2) initial value: the L2 projection onto V_H = V_H1 + V_H2 is
    the identity on V_H, so u0 = Psi1 a + Psi2 b comes back as (a, b)."""
    fp, spc, red = run24.fp, run24.spc, run24.red
    rng = np.random.default_rng(23)
    for _ in range(3):
        a = rng.normal(size=red.d1)
        b = rng.normal(size=red.d2)
        u0 = fp.to_nodal(spc.Psi1 @ a + spc.Psi2 @ b)
        ga, gb = red.project_initial(u0)
        assert np.abs(ga - a).max() <= 1e-9 * np.abs(a).max()
        assert np.abs(gb - b).max() <= 1e-9 * np.abs(b).max()
        # the projected function itself to 1e-12
        back = spc.Psi1 @ ga + spc.Psi2 @ gb
        assert np.linalg.norm(back - fp.to_interior(u0)) <= 1e-12 * np.linalg.norm(back)


def test_initial_projection_residual_is_l2_orthogonal_to_v_h(run24):
    """For u0 outside V_H the residual u0 - Pi u0 is M_f-orthogonal to every
    basis of V_H1 and of V_H2 (Galerkin orthogonality)."""
    fp, spc, red = run24.fp, run24.spc, run24.red
    rng = np.random.default_rng(29)
    u0 = np.zeros((fp.n_f + 1) ** 2)
    u0[fp.interior] = rng.normal(size=fp.D)
    a, b = red.project_initial(u0)
    r = fp.to_interior(u0) - spc.Psi1 @ a - spc.Psi2 @ b
    Mr = fp.M @ r
    scale = np.abs(fp.M @ fp.to_interior(u0)).sum()
    assert np.abs(spc.Psi1.T @ Mr).max() <= 1e-10 * scale
    assert np.abs(spc.Psi2.T @ Mr).max() <= 1e-10 * scale


def _semi_discrete(red, x0, t):
    """Exact solution of M_H x' + A_H x = 0 at time t (the method of lines in
    V_H without time discretisation), by the eigendecomposition of the
    symmetric pencil (A_H, M_H)."""
    lam, V = sla.eigh(red.AH(), red.MH())
    return V @ (np.exp(-lam * t) * (V.T @ (red.MH() @ x0)))


def test_closed_form_first_order_in_dt_and_convergent_under_refinement():
    """kappa = 1, f = 0, u0 = sin(pi x) sin(pi y): u = exp(-2 pi^2 t) u0.
    (i) At a fixed space, the splitting scheme eqs. (2.4)-(2.5) converges to
    the semi-discrete solution with order 1 in dt (observed rates of the
    dt-halving sequence in [0.8, 1.2]).  (ii) Refining the fine grid, the
    coarse grid, the oversampling and dt together, the error against the
    closed form decreases, by more than a factor 2 per level.  The
    oversampling grows with the level (ell = 1, 2, 3): the localised CEM
    bases of Section 3.1 need ell ~ log(1/H) layers, and with ell fixed the
    error grows as H shrinks (kappa = 1, J = 2, ell = 2: 1.5e-2, 4.2e-2,
    1.8e-1 at H = 1/4, 1/8, 1/16).  dt shrinks like H^2, which keeps
    dt lambda_max(A22, M22) at 0.10 on every level (the explicit V_H2 step of
    eq. (2.5) needs dt ~ H^2)."""
    T = 0.02
    # (i) order in dt on one space
    prob = config_small(n_f=32, nc=8, J=2, ell=2, N=1, P=8, channels=0, contrast=1.0, u0_kind="sin",
                        f_kind="zero")
    o = OracleRun(prob, T=T)
    x0 = np.concatenate([o.u0, o.w0])
    ex = _semi_discrete(o.red, x0, T)
    errs = []
    z1, z2 = np.zeros(o.red.d1), np.zeros(o.red.d2)
    for P in (16, 32, 64, 128):
        sch = Scheme(o.red, T, 1, P, 0.1)
        u, w = sch.F_seq(o.u0, o.w0, z1, z2)
        d = np.concatenate([u, w]) - ex
        errs.append(np.sqrt(d @ o.red.MH() @ d))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 0.8) & (rates < 1.2)), rates
    # (ii) joint refinement against the closed form
    tot = []
    for n_f, ell, P in ((16, 1, 16), (32, 2, 64), (64, 3, 256)):
        prob = config_small(n_f=n_f, nc=n_f // 8, J=3, ell=ell, N=1, P=P, channels=0, contrast=1.0,
                            u0_kind="sin", f_kind="zero")
        o = OracleRun(prob, T=T)
        assert T / P * o.lam22 < 0.2
        u, w = Scheme(o.red, T, 1, P, 0.1).F_seq(o.u0, o.w0, np.zeros(o.red.d1), np.zeros(o.red.d2))
        uh = o.red.prolong(u, w)
        x = np.arange(n_f + 1) / n_f
        X, Y = np.meshgrid(x, x)
        exact = np.exp(-2 * np.pi ** 2 * T) * (np.sin(np.pi * X) * np.sin(np.pi * Y)).ravel()
        tot.append(np.linalg.norm(uh - exact) / np.linalg.norm(exact))
    assert tot[0] < 0.05 and tot[1] < 0.5 * tot[0] and tot[2] < 0.5 * tot[1], tot


def _window_constraints(fp, spc, win, weighted):
    """Constraint rows of eq. (3.2) on a window: the indicator rows either
    kappa_tilde-weighted (the oracle's reading) or plain integrals over the
    continuum (eq. (3.6) as printed), and the enrichment rows; with the
    right-hand side of the target block's constraints."""
    loc = -np.ones((fp.n_f + 1) ** 2, dtype=int)
    loc[win.gid] = np.arange(win.gid.size)
    h = 1.0 / fp.n_f
    rows, gram = [], []
    for key in win.blocks:
        blk = spc.blocks[key]
        li = loc[blk.gid]
        n_ind = blk.R.shape[0]
        for q in range(blk.con_rows.shape[0]):
            full = blk.con_rows[q].copy()
            g = blk.con_gram[q]
            if q < n_ind and not weighted:
                # plain integral of phi over the continuum's cells: a bilinear
                # function integrates to h^2 / 4 times the sum of its corners
                full = np.zeros(blk.nb)
                area = 0.0
                for c in np.nonzero(_continuum_cells(fp, blk, q))[0]:
                    full[blk.corners[c]] += h * h / 4.0
                    area += h * h
                g = area
            row = np.zeros(win.gid.size)
            row[li[li >= 0]] = full[li >= 0]
            rows.append(row)
            gram.append((key, q, g))
    return np.array(rows), gram


def _continuum_cells(fp, blk, q):
    """Boolean mask of the block's cells forming its q-th continuum (matrix
    first when present, then the 4-connected high-conductivity components in
    order of their smallest cell), recomputed from kappa."""
    from oracle.spaces import components
    kap = fp.kappa[blk.by * blk.bs:(blk.by + 1) * blk.bs, blk.bx * blk.bs:(blk.bx + 1) * blk.bs]
    matrix = kap == fp.kappa.min()
    conts = []
    if matrix.any():
        conts.append(np.nonzero(matrix.ravel())[0])
    conts.extend(np.array(c) for c in components(~matrix))
    m = np.zeros(kap.size, dtype=bool)
    m[conts[q]] = True
    return m


def _dense_cem(fp, win, C, rhs_row_index, rhs_values):
    """min a(phi, phi) subject to C phi = e (dense KKT, numpy solve)."""
    Aw = fp.A_full[win.gid][:, win.gid].toarray()
    m = C.shape[0]
    K = np.block([[Aw, C.T], [C, np.zeros((m, m))]])
    out = []
    for r, v in zip(rhs_row_index, rhs_values):
        b = np.zeros(Aw.shape[0] + m)
        b[Aw.shape[0] + r] = v
        out.append(np.linalg.solve(K, b)[:Aw.shape[0]])
    return np.array(out).T


@pytest.mark.parametrize("uniform", [True, False])
def test_weighted_and_plain_continuum_constraints(uniform):
    """eq. (3.6) prints the NLMC constraints as plain integrals over each
    continuum; the oracle weights them by kappa_tilde.  Where kappa is
    constant on every continuum (every workload here: channels and inclusions
    of one value) the two give the same bases; a channel with two kappa
    values is the negative control."""
    prob = config_small(n_f=16, nc=2, J=1, ell=1, N=2, P=4, channels=2, contrast=1e3)
    kappa = prob.kappa.copy()
    if not uniform:
        hi = np.argwhere(kappa > 1.0)
        y, x = hi[len(hi) // 2]
        kappa[y, x] = 10.0 * kappa.max()        # two values inside one channel
    from oracle.spaces import Spaces
    fp = FineProblem(prob.n_f, kappa, prob.nc)
    spc = Spaces(fp, prob.J, prob.ell, workers=1)
    win = Window(fp, 0, 0, prob.ell)
    phi = cem_window(fp, spc.blocks, win, (0, 0))
    Cw, gw = _window_constraints(fp, spc, win, weighted=True)
    Cp, gp = _window_constraints(fp, spc, win, weighted=False)
    tgt = [i for i, (key, q, g) in enumerate(gw) if key == (0, 0)]
    # brute force with the weighted rows reproduces the oracle's sparse solve
    pw = _dense_cem(fp, win, Cw, tgt, [gw[i][2] for i in tgt])
    assert np.abs(pw - phi).max() <= 1e-8 * np.abs(phi).max()
    # plain integrals: the right-hand side is the continuum's area
    pp = _dense_cem(fp, win, Cp, tgt, [gp[i][2] for i in tgt])
    diff = np.abs(pp - phi).max() / np.abs(phi).max()
    if uniform:
        assert diff <= 1e-8, diff
    else:
        assert diff > 1e-4, diff
