"""Pins of the oracle's time stepping, WR propagator and parareal driver.

Each test compares with something fixed outside the oracle's own code path:
brute-force Kronecker solves, the variational form of eqs. (2.4)-(2.5)
evaluated on fine-grid vectors, backward/forward Euler closed forms, the
exact heat solution, the energy bound, and the parareal/WR fixed points.
"""
import types

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fem import FineProblem
from oracle.spaces import Spaces
from oracle.reduced import Reduced, stable_T
from oracle.scheme import Scheme
from oracle import parareal as pr
from oracle.pipeline import OracleRun


@pytest.fixture(scope="module")
def run16(small_problem):
    return OracleRun(small_problem)


def test_split_is_direct_and_structured(run16):
    spc, red = run16.spc, run16.red
    assert red.d1 == spc.Psi1.shape[1] and red.d2 == spc.Psi2.shape[1]
    # direct sum: [Psi1 Psi2] has full column rank and gamma < 1
    sv = np.linalg.svd(np.column_stack([spc.Psi1, spc.Psi2]), compute_uv=False)
    assert sv[-1] > 1e-8 * sv[0]
    assert run16.gamma < 0.99
    # V_H = span of all bases (eq. (3.7) keeps the total space)
    allr = np.linalg.matrix_rank(spc.Psi_all, tol=1e-9 * np.linalg.norm(spc.Psi_all, 2))
    both = np.linalg.matrix_rank(np.column_stack([spc.Psi_all, spc.Psi1, spc.Psi2]),
                                 tol=1e-9 * np.linalg.norm(spc.Psi_all, 2))
    assert allr == both == red.d1 + red.d2
    # psi_tilde are s-orthogonal to psi_bar; the L fracture psi_tilde sum to zero
    S = run16.fp.S
    Sb = S @ spc.psi_bar
    assert np.abs(Sb @ spc.Psi1).max() < 1e-10 * np.abs(Sb @ spc.Psi_all).max()
    fr = np.nonzero(spc.kind == 1)[0]
    c = (Sb @ spc.Psi_all[:, fr]) / (spc.psi_bar @ Sb)
    tilde_all = spc.Psi_all[:, fr] - np.outer(spc.psi_bar, c)
    assert np.abs(tilde_all.sum(axis=1)).max() < 1e-11 * np.abs(tilde_all).max()


def test_cem_constraints_and_minimality(run16):
    from oracle.spaces import Window, cem_window
    fp, spc = run16.fp, run16.spc
    win = Window(fp, 1, 2, spc.ell)
    phi = cem_window(fp, spc.blocks, win, (1, 2))
    loc = -np.ones((fp.n_f + 1) ** 2, dtype=int)
    loc[win.gid] = np.arange(win.gid.size)
    Cr = []
    for key in win.blocks:
        blk = spc.blocks[key]
        li = loc[blk.gid]
        for q in range(blk.con_rows.shape[0]):
            row = np.zeros(win.gid.size)
            row[li[li >= 0]] = blk.con_rows[q, li >= 0]
            Cr.append(row)
    C = np.array(Cr)
    # constraints s(phi, nu) = s(psi, nu): a unit-Gram-weighted row on the target
    t = spc.blocks[(1, 2)]
    got = C @ phi
    start = [k for k in win.blocks].index((1, 2))
    off = sum(spc.blocks[k].con_rows.shape[0] for k in win.blocks[:start])
    want = np.zeros_like(got)
    for q in range(t.con_rows.shape[0]):
        want[off + q, q] = t.con_gram[q]
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    # energy minimality: the gradient A phi lies in range(C^T) (brute-force least squares)
    Aw = fp.A_full[win.gid][:, win.gid].toarray()
    g = Aw @ phi
    coef, *_ = np.linalg.lstsq(C.T, g, rcond=None)
    assert np.abs(C.T @ coef - g).max() < 1e-8 * np.abs(g).max()


def _variational_step(fp, P1, P2, u, w, ul, wl, h, b):
    """eqs. (2.4)-(2.5) written on fine-grid vectors: find c1, c2 with
    u' = P1 c1, w' = P2 c2 such that for every basis test function v1 of V_H1
    and v2 of V_H2 the two identities hold ((.,.) = M_f, a = A_f)."""
    M, A = fp.M.toarray(), fp.A.toarray()
    d1 = P1.shape[1]
    # eq. (2.4): (u'-u, v1)/h + (w-wl, v1)/h + a(u' + w, v1) = (f, v1)
    L1 = P1.T @ (M / h + A) @ P1
    r1 = P1.T @ (M @ u / h - M @ (w - wl) / h - A @ w + b)
    c1 = np.linalg.solve(L1, r1)
    un = P1 @ c1
    # eq. (2.5): (w'-w, v2)/h + (u-ul, v2)/h + a(u' + w, v2) = (f, v2)
    L2 = P2.T @ (M / h) @ P2
    r2 = P2.T @ (M @ w / h - M @ (u - ul) / h - A @ (un + w) + b)
    c2 = np.linalg.solve(L2, r2)
    return c1, c2


def test_step_matches_variational_form(run16):
    fp, spc, red = run16.fp, run16.spc, run16.red
    sch = run16.sch
    rng = np.random.default_rng(5)
    cu, cw, cul, cwl = (rng.normal(size=red.d1), rng.normal(size=red.d2),
                        rng.normal(size=red.d1), rng.normal(size=red.d2))
    P1, P2 = spc.Psi1, spc.Psi2
    b = fp.load(rng.normal(size=(fp.n_f + 1) ** 2))
    F1, F2 = P1.T @ b, P2.T @ b
    h = sch.dt
    ref1, ref2 = _variational_step(fp, P1, P2, P1 @ cu, P2 @ cw, P1 @ cul, P2 @ cwl, h, b)
    got1, got2 = sch.step(cu, cw, cul, cwl, h, F1, F2, sch.cho_f)
    assert np.allclose(got1, ref1, rtol=1e-9, atol=1e-10 * np.abs(ref1).max())
    assert np.allclose(got2, ref2, rtol=1e-9, atol=1e-10 * np.abs(ref2).max())


def _decoupled(d1=5, d2=4, seed=1):
    rng = np.random.default_rng(seed)
    def spd(n):
        X = rng.normal(size=(n, n))
        return X @ X.T + n * np.eye(n)
    r = types.SimpleNamespace()
    r.M11, r.A11, r.M22, r.A22 = spd(d1), spd(d1), spd(d2), spd(d2) * 0.1
    r.M12 = np.zeros((d1, d2)); r.A12 = np.zeros((d1, d2))
    r.M21, r.A21 = r.M12.T, r.A12.T
    r.d1, r.d2 = d1, d2
    return r


def test_decoupled_split_reduces_to_backward_and_forward_euler():
    # M12 = A12 = 0: eq. (2.4) is backward Euler (eq. (2.3)) in V_H1 and
    # eq. (2.5) is forward Euler in V_H2
    r = _decoupled()
    sch = Scheme(r, T=0.3, N=3, P=5, alpha=0.1)
    rng = np.random.default_rng(2)
    u0, w0 = rng.normal(size=r.d1), rng.normal(size=r.d2)
    F1, F2 = rng.normal(size=r.d1), rng.normal(size=r.d2)
    u, w = sch.F_seq(u0, w0, F1, F2)
    ub, wf = u0.copy(), w0.copy()
    for _ in range(5):
        ub = np.linalg.solve(r.M11 + sch.dt * r.A11, r.M11 @ ub + sch.dt * F1)
        wf = wf + sch.dt * np.linalg.solve(r.M22, F2 - r.A22 @ wf)
    assert np.allclose(u, ub, rtol=1e-12) and np.allclose(w, wf, rtol=1e-12)


def test_alpha_circulant_diagonalisation_matches_dense_kron():
    r = _decoupled(d1=6, d2=2)
    for P, alpha in [(5, 0.1), (8, 0.5), (7, 1e-3)]:
        sch = Scheme(r, T=0.2, N=2, P=P, alpha=alpha)
        # eq. (4.5): B = S D S^-1 with S = Lambda V, Lambda = diag(alpha^{-(p-1)/P})
        B = sch.B_matrix()
        Lam = np.diag(alpha ** (-np.arange(P) / P))
        V = np.exp(2j * np.pi * np.outer(np.arange(P), np.arange(P)) / P)   # inverse-DFT columns
        S = Lam @ V
        assert np.allclose(S @ np.diag(sch.dk) @ np.linalg.inv(S), B, atol=1e-9 * np.abs(B).max())
        rng = np.random.default_rng(P)
        Fv = rng.normal(size=(P, r.d1))
        K = np.kron(B, r.M11) + np.kron(np.eye(P), r.A11)
        ref = np.linalg.solve(K, Fv.ravel()).reshape(P, r.d1)
        got = sch.all_at_once_solve(Fv)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_wr_fixed_point_is_sequential_scheme(run16):
    sch = run16.sch
    red = run16.red
    rng = np.random.default_rng(11)
    starts = [(rng.normal(size=red.d1), rng.normal(size=red.d2)) for _ in range(3)]
    F1s = [run16.F1 * a for a in (0.5, 1.0, 2.0)]
    F2s = [run16.F2 * a for a in (0.5, 1.0, 2.0)]
    hist = []
    ends, it = sch.F_wr(starts, F1s, F2s, wr_tol=1e-13, wr_max=300, history=hist)
    for n in range(3):
        us, ws = sch.F_seq(*starts[n], F1s[n], F2s[n])
        scale = max(np.abs(us).max(), np.abs(ws).max())
        assert np.abs(ends[n][0] - us).max() < 1e-11 * scale
        assert np.abs(ends[n][1] - ws).max() < 1e-11 * scale
    # Theorem 4.1: contraction per WR iteration of order gamma^2
    h = np.array(hist)
    rates = h[3:12] / h[2:11]
    assert np.median(rates) < 1.2 * run16.gamma ** 2 + 0.05


def test_parareal_k_equals_N_is_exact(run16):
    # Algorithm 1 reproduces the sequential fine propagation after N sweeps
    u_s, w_s = run16.sequential()
    u, w, st = run16.solve(eps=0.0, k_max=run16.prob.N, fine="seq")
    scale = np.abs(u_s).max()
    assert st["K1"] == run16.prob.N
    assert np.abs(u - u_s).max() < 1e-12 * scale and np.abs(w - w_s).max() < 1e-12 * scale
    # ... and states n <= k are exact after k sweeps
    u2, w2, _ = run16.solve(eps=0.0, k_max=2, fine="seq")
    assert np.abs(u2[:3] - u_s[:3]).max() < 1e-12 * scale
    # with the WR fine propagator the limit is reached to the WR tolerance
    u3, w3, st3 = run16.solve(eps=0.0, k_max=run16.prob.N, wr_tol=1e-14, wr_max=400)
    assert np.abs(u3 - u_s).max() < 1e-10 * scale


def test_parareal_jumps_contract(run16):
    _, _, st = run16.solve(eps=1e-14, fine="seq")
    j = np.array(st["jumps"])
    assert np.all(j[1:] < j[:-1])


def test_energy_bound_and_negative_control(run16):
    # derived from eqs. (2.4)-(2.5) with v1 = u_{n+1}-u_n, v2 = w_{n+1}-w_n, f = 0:
    # E_n = 1/2 ||u_n + w_n||_a^2 + gamma/(2 h) (||u_n-u_{n-1}||^2 + ||w_n-w_{n-1}||^2)
    # is non-increasing whenever h lambda_max(A22, M22) <= 2 (1 - gamma)
    red, g, lam = run16.red, run16.gamma, run16.lam22
    AH, MH = red.AH(), red.MH()
    rng = np.random.default_rng(4)
    u, w = rng.normal(size=red.d1), rng.normal(size=red.d2)

    def energies(h, steps):
        sch = Scheme(red, T=h * steps, N=1, P=steps, alpha=0.1)
        _, _, traj = sch.F_seq(u, w, np.zeros(red.d1), np.zeros(red.d2), return_traj=True)
        E = []
        for n in range(1, len(traj)):
            z = np.concatenate(traj[n])
            dz = np.concatenate([traj[n][0] - traj[n - 1][0], np.zeros(red.d2)])
            du = traj[n][0] - traj[n - 1][0]
            dw = traj[n][1] - traj[n - 1][1]
            e = 0.5 * z @ AH @ z + g / (2 * h) * (du @ red.M11 @ du + dw @ red.M22 @ dw)
            E.append(e)
        return np.array(E)

    h_ok = 0.95 * 2 * (1 - g) / lam
    E = energies(h_ok, 40)
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    E_bad = energies(8.0 / lam, 40)
    assert E_bad[-1] > 10 * E_bad[0]


def test_closed_form_heat_decay():
    # kappa = 1, f = 0, u0 = sin(pi x) sin(pi y): u = exp(-2 pi^2 t) u0 (eq. (2.1))
    from paper_2411_09244_gb300.inputs import config_small
    errs = []
    for n_f, P in [(16, 8), (32, 16)]:
        prob = config_small(n_f=n_f, nc=4, J=2, ell=2, N=4, P=P, channels=0, contrast=1.0,
                            u0_kind="sin", f_kind="zero")
        T = 0.02
        o = OracleRun(prob, T=T)
        u, w = o.sequential()
        uh = o.red.prolong(u[-1], w[-1])
        x = np.arange(n_f + 1) / n_f
        X, Y = np.meshgrid(x, x)
        exact = np.exp(-2 * np.pi ** 2 * T) * (np.sin(np.pi * X) * np.sin(np.pi * Y)).ravel()
        errs.append(np.linalg.norm(uh - exact) / np.linalg.norm(exact))
    assert errs[1] < errs[0] < 0.05


def test_backward_euler_16x16_brute_force_reference():
    # full-Q1 backward Euler eq. (2.3) on 16x16 is the spatial reference; the
    # multiscale splitting solution approaches it, and more oversampling
    # layers (Section 3.1) bring it closer
    from paper_2411_09244_gb300.inputs import config_small
    rel = {}
    for ell in (1, 2):
        prob = config_small(n_f=16, nc=4, J=3, ell=ell, N=4, P=8, channels=2, contrast=1e3,
                            u0_kind="zero", f_kind="ones")
        o = OracleRun(prob)
        fp = o.fp
        dt = o.sch.dt
        A, M = fp.A.toarray(), fp.M.toarray()
        b = fp.load(prob.f)
        x = np.zeros(fp.D)
        for n in range(prob.N):
            for _ in range(prob.P):
                x = np.linalg.solve(M + dt * A, M @ x + dt * prob.amp[n] * b)
        u, w = o.sequential()
        uh = fp.to_interior(o.red.prolong(u[-1], w[-1]))
        rel[ell] = np.linalg.norm(uh - x) / np.linalg.norm(x)
    assert rel[2] < 0.1 and rel[2] < 0.5 * rel[1]


def test_stable_T_two_significant_digits():
    assert stable_T(10, 0.5, 1000.0) == pytest.approx(0.0067)
    assert stable_T(8, 0.0, 1.0) == pytest.approx(7.2)
