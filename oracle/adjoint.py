"""Adjoint of the limit of Algorithm 1 for an observation misfit (oracle).

The paper does not treat differentiation.  Reading: differentiate the map
that Algorithm 1 converges to, u_h* = the fine scheme of eqs. (2.4)-(2.5)
run interval after interval with the lag terms restarted at each coarse
boundary, not a tolerance-dependent iterate.  With the state x_n = (u_n, w_n)
at the coarse times and the source amp[n] * f_shape on interval n,

    x_0     = M_H^-1 [Psi1 Psi2]^T M_f u0          (the projection of eq. (2.2))
    x_{n+1} = Phi x_n + amp[n] s,   n = 0..N-1,

where Phi is the interval map of the fine scheme with zero source and s its
response to the unit source from a zero state (the operator is the same on
every interval).  The misfit over observation nodes o at t_1..t_N,

    J = 1/2 sum_{n=1..N} sum_o ((Psi x_n)(o) - d_{o,n})^2 = 1/2 sum_n ||O x_n - d_n||^2,

is quadratic in (u0, amp).  Its gradient by the backward recurrence

    lambda_N = O^T r_N,  lambda_n = Phi^T lambda_{n+1} + O^T r_n (n = N-1..1),
    lambda_0 = Phi^T lambda_1,   r_n = O x_n - d_n,
    dJ/d amp[n] = <lambda_{n+1}, s>,
    dJ/d u0     = M_f [Psi1 Psi2] M_H^-1 lambda_0   (M_f, M_H symmetric).

Phi^T is applied step by step with the transpose of the one-step map of the
scheme.  The step is linear in the augmented state z = (u, w, u_lag, w_lag);
its matrix S is formed column by column from Scheme.step itself, so the
transpose is that of the scheme exactly as the oracle defines it.  The
interval map is Phi = E_out S^P E_in with E_in x = (u, w, u, w) (lag restart)
and E_out z = (u, w), hence Phi^T = E_in^T (S^T)^P E_out^T.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


class Adjoint:
    def __init__(self, run, obs_nodes):
        """run: pipeline.OracleRun; obs_nodes: node ids (x fastest, all nodes)."""
        self.run = run
        red = run.red
        self.d1, self.d2 = red.d1, red.d2
        self.d = self.d1 + self.d2
        # observation operator: rows of [Psi1 Psi2] at the observation nodes
        pos = {int(k): i for i, k in enumerate(run.fp.interior)}
        rows = [pos[int(k)] for k in obs_nodes]
        self.O = np.hstack([red.spc.Psi1, red.spc.Psi2])[rows, :]
        self._S = None
        self._s = None

    # -- the scheme's one-step matrix and unit-source response ---------------
    def step_matrix(self):
        """S (2d x 2d) with z' = S z for one fine step without source."""
        if self._S is None:
            sch = self.run.sch
            d1, d2, d = self.d1, self.d2, self.d
            z1, z2 = np.zeros(d1), np.zeros(d2)
            S = np.zeros((2 * d, 2 * d))
            for j in range(2 * d):
                e = np.zeros(2 * d)
                e[j] = 1.0
                u, w, ul, wl = e[:d1], e[d1:d], e[d:d + d1], e[d + d1:]
                u1, w1 = sch.step(u, w, ul, wl, sch.dt, z1, z2, sch.cho_f)
                S[:, j] = np.concatenate([u1, w1, u, w])
            self._S = S
        return self._S

    def unit_response(self):
        """s = F*(0; F1, F2): the interval's response to the unit-amplitude
        source from a zero state (Scheme.F_seq)."""
        if self._s is None:
            r = self.run
            u, w = r.sch.F_seq(np.zeros(self.d1), np.zeros(self.d2), r.F1, r.F2)
            self._s = np.concatenate([u, w])
        return self._s

    def step_source(self):
        """c: the source term of one fine step (unit amplitude, zero state)."""
        r, sch = self.run, self.run.sch
        u1, w1 = sch.step(np.zeros(self.d1), np.zeros(self.d2), np.zeros(self.d1), np.zeros(self.d2),
                          sch.dt, r.F1, r.F2, sch.cho_f)
        return np.concatenate([u1, w1, np.zeros(self.d)])

    # -- interval map and its transpose ---------------------------------------
    def Phi(self, x):
        S = self.step_matrix()
        z = np.concatenate([x, x])                      # E_in: lag restart
        for _ in range(self.run.sch.P):
            z = S @ z
        return z[:self.d]                               # E_out

    def Phi_T(self, lam):
        S = self.step_matrix()
        z = np.concatenate([lam, np.zeros(self.d)])     # E_out^T
        for _ in range(self.run.sch.P):
            z = S.T @ z
        return z[:self.d] + z[self.d:]                  # E_in^T

    # -- forward map, misfit, gradient ---------------------------------------
    def initial_state(self, u0_nodal):
        u, w = self.run.red.project_initial(u0_nodal)
        return np.concatenate([u, w])

    def forward(self, u0_nodal, amp):
        """Coarse states x_0..x_N of u_h* (sequential fine scheme)."""
        r = self.run
        u0, w0 = r.red.project_initial(u0_nodal)
        from .parareal import sequential_fine
        U, W = sequential_fine(r.sch, u0, w0, r.F1, r.F2, np.asarray(amp, dtype=np.float64))
        return np.hstack([U, W])

    def observe(self, X):
        """[N, n_obs]: u_h(x_o, t_n) for n = 1..N."""
        return X[1:] @ self.O.T

    def misfit(self, u0_nodal, amp, data):
        R = self.observe(self.forward(u0_nodal, amp)) - data
        return 0.5 * float(np.sum(R * R))

    def gradient(self, u0_nodal, amp, data, amp_mode="response"):
        """(J, dJ/du0 [(n_f+1)^2], dJ/damp [N]).  amp_mode "response" uses
        <lambda_{n+1}, s>; "recompute" accumulates sum_p <mu_p, c> with the
        adjoint recomputed step by step inside each interval."""
        red, fp = self.run.red, self.run.fp
        N, P, d = self.run.sch.N, self.run.sch.P, self.d
        X = self.forward(u0_nodal, amp)
        R = self.observe(X) - data                       # r_1..r_N
        J = 0.5 * float(np.sum(R * R))
        lam = [None] * (N + 1)
        lam[N] = self.O.T @ R[N - 1]
        for n in range(N - 1, 0, -1):
            lam[n] = self.Phi_T(lam[n + 1]) + self.O.T @ R[n - 1]
        lam[0] = self.Phi_T(lam[1])
        g_amp = np.zeros(N)
        if amp_mode == "response":
            s = self.unit_response()
            for n in range(N):
                g_amp[n] = lam[n + 1] @ s
        else:
            S, c = self.step_matrix(), self.step_source()
            for n in range(N):
                z = np.concatenate([lam[n + 1], np.zeros(d)])
                acc = 0.0
                for _ in range(P):                       # mu_P, mu_{P-1}, ..., mu_1
                    acc += z @ c
                    z = S.T @ z
                g_amp[n] = acc
        y = np.linalg.solve(red.MH(), lam[0])
        g_u0 = fp.M_full @ fp.to_nodal(red.spc.Psi1 @ y[:self.d1] + red.spc.Psi2 @ y[self.d1:])
        return J, np.asarray(g_u0).ravel(), g_amp
