"""Reduced (Galerkin) operators and scalar diagnostics.

eq. (3.8): M_ij = Psi_i^T M_f Psi_j, A_ij = Psi_i^T A_f Psi_j, F_i = Psi_i^T f
(read as Psi_i^T M_f f, see fem.FineProblem.load).

gamma, eq. (4.15): the largest cosine between V_H1 and V_H2 in L2,
gamma^2 = lambda_max(M12 M22^-1 M21, M11).

Time-step condition of Section 3.2 (after eq. (3.7)):
Delta t * sup_{v in V_H2} ||v||_a^2 / ||v||^2 <= 1 - gamma^2, with the sup
equal to lambda_max(A22, M22).

Initial value u_{H,0}, eq. (2.2): the L2 projection of u0 onto V_H, solved
through the joint Gram matrix M_H = [[M11, M12], [M21, M22]] and split into
(u_0, w_0) (reading of "projected onto corresponding subspaces" after
eq. (2.5): two separate projections onto non-orthogonal subspaces would not
reproduce u0 even when u0 lies in V_H).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .fem import FineProblem
from .spaces import Spaces


class Reduced:
    def __init__(self, fp: FineProblem, spc: Spaces):
        P1, P2 = spc.Psi1, spc.Psi2
        M, A = fp.M, fp.A
        self.M11 = P1.T @ (M @ P1)
        self.A11 = P1.T @ (A @ P1)
        self.M22 = P2.T @ (M @ P2)
        self.A22 = P2.T @ (A @ P2)
        self.M12 = P1.T @ (M @ P2)
        self.A12 = P1.T @ (A @ P2)
        self.M21 = self.M12.T
        self.A21 = self.A12.T
        self.d1, self.d2 = P1.shape[1], P2.shape[1]
        self.fp = fp
        self.spc = spc

    def MH(self):
        return np.block([[self.M11, self.M12], [self.M21, self.M22]])

    def AH(self):
        return np.block([[self.A11, self.A12], [self.A21, self.A22]])

    def load(self, f_nodal):
        b = self.fp.load(f_nodal)
        return self.spc.Psi1.T @ b, self.spc.Psi2.T @ b

    def gamma(self) -> float:
        X = self.M12 @ np.linalg.solve(self.M22, self.M21)
        lam = sla.eigh(0.5 * (X + X.T), self.M11, eigvals_only=True)
        return float(math.sqrt(max(lam[-1], 0.0)))

    def lambda_max_22(self) -> float:
        return float(sla.eigh(self.A22, self.M22, eigvals_only=True)[-1])

    def project_initial(self, u0_nodal):
        g = self.fp.to_interior(self.fp.M_full @ np.asarray(u0_nodal, dtype=np.float64))
        rhs = np.concatenate([self.spc.Psi1.T @ g, self.spc.Psi2.T @ g])
        c = np.linalg.solve(self.MH(), rhs)
        return c[:self.d1], c[self.d1:]

    def prolong(self, u, w):
        """u_h = Psi1 u + Psi2 w on all nodes (zero on the boundary)."""
        return self.fp.to_nodal(self.spc.Psi1 @ u + self.spc.Psi2 @ w)


def stable_T(N: int, gamma: float, lam_max22: float, T_cap: float | None = None) -> float:
    """Final time whose coarse step satisfies the condition of Section 3.2
    with margin 0.9: T = 0.9 N (1 - gamma^2) / lambda_max(A22, M22), rounded
    down to two significant digits (so that two independent computations of
    gamma and lambda_max agree on T)."""
    t = 0.9 * N * (1.0 - gamma * gamma) / lam_max22
    e = math.floor(math.log10(t)) - 1
    t = math.floor(t / 10.0 ** e) * 10.0 ** e
    if T_cap is not None:
        t = min(t, T_cap)
    return t
