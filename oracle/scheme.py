"""Time stepping in V_H1 x V_H2, original (basis) coordinates.

Partially explicit splitting scheme, eqs. (2.4)-(2.5), in matrix form for a
step h from (u_n, w_n) with lags (u_{n-1}, w_{n-1}):

  (M11 + h A11) u_{n+1} = M11 u_n - M12 (w_n - w_{n-1}) - h A12 w_n + h F1
  M22 w_{n+1}           = M22 w_n - M21 (u_n - u_{n-1}) - h (A21 u_{n+1} + A22 w_n) + h F2

Readings: the source is taken at t_{n+1} (as in eqs. (2.3), (4.8), (4.9));
every propagator call (G over one coarse step, F over one interval) restarts
with zero lag increments, u_{-1} = u_0 and w_{-1} = w_0, so the parareal state
is exactly (u_n, w_n) as Algorithm 1 propagates it.  A source that is
f_shape * amp[n] on interval n gives F1 = amp[n] * Psi1^T M_f f_shape.

Fine propagator F: the waveform relaxation of Section 4.2, eqs. (4.8)-(4.13),
with P steps of dt = Delta t / P on each interval:
  * V_H1 part: the all-at-once system (B (x) M11 + I (x) A11) U^j = F~
    (eq. (4.12)) with B the alpha-circulant matrix of eq. (4.4), solved by
    the diagonalisation B = S D S^-1, S = Lambda V (eqs. (4.5)-(4.7)):
    (a) scale by Lambda^-1 and FFT over the time index, (b) one complex
    shifted solve (d_k M11 + A11) q_k = p_k per frequency, (c) inverse FFT
    and scale by Lambda.
  * right-hand side (reading of the garbled display after eq. (4.12)):
    f~^p = F1 - (1/dt) M12 (w_{p-1} - w_{p-2}) - A12 w_{p-1}, p = 1..P, with
    w_{-1} := w_0 and W from the previous WR iterate; at p = 1 the periodic-
    like initial condition U^j(0) = u_0 + alpha (u_P^j - u_P^{j-1}) adds
    (1/dt) M11 (u_0 - alpha u_P^{j-1}).
  * V_H2 part: eq. (4.9) swept sequentially in p with U^j, u_{-1} = u_0.
  * start (silent in the paper): W^0 = w_0 and U^0 = u_0 at every step;
    stop when max over intervals and steps of max(||u_p^j - u_p^{j-1}||_M11,
    ||w_p^j - w_p^{j-1}||_M22) <= wr_tol, or after wr_max iterations.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .reduced import Reduced


class Scheme:
    def __init__(self, red: Reduced, T: float, N: int, P: int, alpha: float):
        self.red = red
        self.T, self.N, self.P, self.alpha = T, N, P, alpha
        self.Dt = T / N
        self.dt = self.Dt / P
        r = red
        self.cho_G = sla.cho_factor(r.M11 + self.Dt * r.A11)
        self.cho_f = sla.cho_factor(r.M11 + self.dt * r.A11)
        self.cho_22 = sla.cho_factor(r.M22)
        # frequency shifts of the alpha-circulant matrix, eq. (4.5)
        beta = alpha ** (1.0 / P)
        self.beta = beta
        k = np.arange(P)
        self.dk = (1.0 - beta * np.exp(-2j * np.pi * k / P)) / self.dt
        self._lu = None

    # -- one step of eqs. (2.4)-(2.5) ---------------------------------------
    def step(self, u, w, u_lag, w_lag, h, F1, F2, cho):
        r = self.red
        rhs_u = r.M11 @ u - r.M12 @ (w - w_lag) - h * (r.A12 @ w) + h * F1
        u1 = sla.cho_solve(cho, rhs_u)
        rhs_w = r.M22 @ w - r.M21 @ (u - u_lag) - h * (r.A21 @ u1 + r.A22 @ w) + h * F2
        w1 = sla.cho_solve(self.cho_22, rhs_w)
        return u1, w1

    def G(self, u, w, F1, F2):
        """Coarse propagator: one step of size Delta t, lags restarted."""
        return self.step(u, w, u, w, self.Dt, F1, F2, self.cho_G)

    def F_seq(self, u, w, F1, F2, return_traj=False):
        """Sequential fine scheme over one interval (the WR fixed point)."""
        ul, wl = u, w
        traj = [(u, w)]
        for _ in range(self.P):
            u1, w1 = self.step(u, w, ul, wl, self.dt, F1, F2, self.cho_f)
            ul, wl, u, w = u, w, u1, w1
            traj.append((u, w))
        return (u, w, traj) if return_traj else (u, w)

    # -- all-at-once V_H1 solve, eq. (4.12) by eq. (4.7) ----------------------
    def _shift_lu(self):
        if self._lu is None:
            r = self.red
            self._lu = [sla.lu_factor(d * r.M11 + r.A11) for d in self.dk]
        return self._lu

    def all_at_once_solve(self, Fv):
        """Solve (B (x) M11 + I (x) A11) U = Fv, Fv [P, d1] real, by steps
        (a)-(c) of eq. (4.7)."""
        P = self.P
        lam_inv = self.beta ** np.arange(P)          # Lambda^-1 diagonal
        Pa = np.fft.fft(lam_inv[:, None] * Fv, axis=0)           # (a)
        Qb = np.empty_like(Pa)
        for k, lu in enumerate(self._shift_lu()):                 # (b)
            Qb[k] = sla.lu_solve(lu, Pa[k])
        U = np.fft.ifft(Qb, axis=0) / lam_inv[:, None]           # (c)
        return U.real

    def B_matrix(self):
        """Dense alpha-circulant B of eq. (4.4) with step dt."""
        P = self.P
        B = np.eye(P) - np.eye(P, k=-1)
        B[0, P - 1] = -self.alpha
        return B / self.dt

    def F_wr(self, starts, F1s, F2s, wr_tol, wr_max, history=None):
        """WR fine propagator on all intervals at once.

        starts: list of (u_0, w_0) per interval; F1s, F2s per interval.
        Returns (ends, iterations)."""
        r = self.red
        P, dt, al = self.P, self.dt, self.alpha
        Nn = len(starts)
        W = [np.tile(w0, (P + 1, 1)) for (_, w0) in starts]     # w_0..w_P
        U = [np.tile(u0, (P + 1, 1)) for (u0, _) in starts]     # u_0..u_P
        it = 0
        for it in range(1, wr_max + 1):
            dmax = 0.0
            for n in range(Nn):
                u0, w0 = starts[n]
                Wp = W[n]
                Fv = np.empty((P, r.d1))
                for p in range(1, P + 1):
                    wm1 = Wp[p - 1]
                    wm2 = Wp[p - 2] if p >= 2 else w0
                    Fv[p - 1] = F1s[n] - (r.M12 @ (wm1 - wm2)) / dt - r.A12 @ wm1
                Fv[0] += r.M11 @ (u0 - al * U[n][P]) / dt
                Unew = np.empty_like(U[n])
                Unew[0] = u0
                Unew[1:] = self.all_at_once_solve(Fv)
                Wnew = np.empty_like(Wp)
                Wnew[0] = w0
                for p in range(P):
                    ulag = Unew[p - 1] if p >= 1 else u0
                    rhs = (r.M22 @ Wnew[p] - r.M21 @ (Unew[p] - ulag)
                           - dt * (r.A21 @ Unew[p + 1] + r.A22 @ Wnew[p]) + dt * F2s[n])
                    Wnew[p + 1] = sla.cho_solve(self.cho_22, rhs)
                du = Unew[1:] - U[n][1:]
                dw = Wnew[1:] - Wp[1:]
                nu = np.sqrt(np.einsum("pi,ij,pj->p", du, r.M11, du))
                nw = np.sqrt(np.einsum("pi,ij,pj->p", dw, r.M22, dw))
                dmax = max(dmax, float(nu.max()), float(nw.max()))
                U[n], W[n] = Unew, Wnew
            if history is not None:
                history.append(dmax)
            if dmax <= wr_tol:
                break
        return [(U[n][P].copy(), W[n][P].copy()) for n in range(Nn)], it
