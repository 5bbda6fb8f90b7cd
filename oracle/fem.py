"""Q1 finite elements on the uniform fine grid of the unit square.

Section 2 poses u_t - div(kappa grad u) = f with homogeneous Dirichlet data
(eq. (2.1)) and discretises it by finite elements in space (eq. (2.2)); the
fine mass and stiffness matrices M_f and A_f are named in Section 3.2 before
eq. (3.8).  The element type is not stated; the reading here is bilinear Q1
on square cells of side h = 1/n_f with kappa constant per cell.

Node numbering: node (i, j), i the x index and j the y index, both 0..n_f,
has id j*(n_f+1) + i.  Cell (ci, cj) has corners in counter-clockwise order
(ci,cj), (ci+1,cj), (ci+1,cj+1), (ci,cj+1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Exact Q1 element matrices on a square (counter-clockwise corners).
# Stiffness of int grad(phi_a).grad(phi_b) (independent of h in 2D).
K_REF = np.array([[4.0, -1.0, -2.0, -1.0],
                  [-1.0, 4.0, -1.0, -2.0],
                  [-2.0, -1.0, 4.0, -1.0],
                  [-1.0, -2.0, -1.0, 4.0]]) / 6.0
# Mass of int phi_a phi_b divided by h^2.
M_REF = np.array([[4.0, 2.0, 1.0, 2.0],
                  [2.0, 4.0, 2.0, 1.0],
                  [1.0, 2.0, 4.0, 2.0],
                  [2.0, 1.0, 2.0, 4.0]]) / 36.0


def cell_corners(n_f: int) -> np.ndarray:
    """[n_f*n_f, 4] node ids of every cell, cells in row-major (y, x) order."""
    ci, cj = np.meshgrid(np.arange(n_f), np.arange(n_f))
    ci = ci.ravel()
    cj = cj.ravel()
    w = n_f + 1
    return np.stack([cj * w + ci, cj * w + ci + 1, (cj + 1) * w + ci + 1, (cj + 1) * w + ci], axis=1)


def assemble(n_f: int, cell_weight_stiff: np.ndarray, cell_weight_mass: np.ndarray):
    """Assemble sum_c w_c K_REF and sum_c v_c h^2 M_REF over all cells, on all
    (n_f+1)^2 nodes (no boundary condition applied).

    Returns (A, M) as CSR matrices."""
    h = 1.0 / n_f
    cor = cell_corners(n_f)
    ws = np.asarray(cell_weight_stiff, dtype=np.float64).ravel()
    wm = np.asarray(cell_weight_mass, dtype=np.float64).ravel()
    rows = np.repeat(cor, 4, axis=1).ravel()
    cols = np.tile(cor, (1, 4)).ravel()
    va = (ws[:, None] * K_REF.ravel()[None, :]).ravel()
    vm = (wm[:, None] * (h * h) * M_REF.ravel()[None, :]).ravel()
    nn = (n_f + 1) ** 2
    A = sp.csr_matrix((va, (rows, cols)), shape=(nn, nn))
    M = sp.csr_matrix((vm, (rows, cols)), shape=(nn, nn))
    A.sum_duplicates()
    M.sum_duplicates()
    return A, M


def interior_nodes(n_f: int) -> np.ndarray:
    """Ids of the (n_f-1)^2 nodes off the boundary (the Dirichlet unknowns)."""
    i, j = np.meshgrid(np.arange(1, n_f), np.arange(1, n_f))
    return (j * (n_f + 1) + i).ravel()


class FineProblem:
    """A_f, M_f on the interior unknowns plus the full-node matrices.

    kappa: [n_f, n_f] cell values (row = y).  The CEM weight of Section 3.1
    is kappa_tilde = kappa * H^-2 (the paper's second option, eq. (3.1)), and
    s(u, v) = int kappa_tilde u v is assembled as the kappa_tilde-weighted Q1
    mass matrix S.
    """

    def __init__(self, n_f: int, kappa: np.ndarray, nc: int):
        self.n_f = n_f
        self.nc = nc
        self.H = 1.0 / nc
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.kappa_tilde = self.kappa / (self.H * self.H)
        ones = np.ones(n_f * n_f)
        self.A_full, self.M_full = assemble(n_f, self.kappa, ones)
        _, self.S_full = assemble(n_f, ones, self.kappa_tilde)
        self.interior = interior_nodes(n_f)
        ix = self.interior
        self.A = self.A_full[ix][:, ix].tocsc()
        self.M = self.M_full[ix][:, ix].tocsc()
        self.S = self.S_full[ix][:, ix].tocsc()
        self.D = ix.size

    def load(self, f_nodal: np.ndarray) -> np.ndarray:
        """Reading of eq. (3.8)'s F = Psi^T f: the load is the Galerkin
        vector (f, phi_a) of the nodal interpolant, b = M_f f on the interior
        rows (the printed F = Psi^T f omits the mass matrix)."""
        return (self.M_full @ np.asarray(f_nodal, dtype=np.float64))[self.interior]

    def to_interior(self, v_nodal: np.ndarray) -> np.ndarray:
        return np.asarray(v_nodal, dtype=np.float64)[self.interior]

    def to_nodal(self, v_int: np.ndarray) -> np.ndarray:
        out = np.zeros((self.n_f + 1) ** 2)
        out[self.interior] = v_int
        return out
