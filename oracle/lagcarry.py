"""Lag-carrying variant of Algorithm 1 (no restart at coarse boundaries).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The scheme of eqs. (2.4)-(2.5) couples each step to the previous one through
the lagged increments u_n - u_{n-1} and w_n - w_{n-1}.  The method restarts
them at every propagator call (u_{-1} = u_0, w_{-1} = w_0 on each interval);
this variant carries them across the coarse boundaries instead, so the fine
solution it converges to is the scheme run uninterrupted over [0, T].

Reading (the paper has no such variant; it is a comparison for the restart
convention): the parareal state becomes x_n = (u_n, w_n, u_n^-, w_n^-), the
states at t_n and one fine step earlier, t_n - dt.
  F(x) : P fine steps from (u, w) with lags (u^-, w^-); returns the end state
         and the state one step before it.
  G(x) : one coarse step of size Delta t whose lag is the fine increment
         extrapolated to the coarse spacing, x - (Delta t / dt)(x - x^-), and
         whose output lag is the linear interpolation x'^- = x' - (dt /
         Delta t)(x' - x) between input and output.  With P = 1 both are
         exact, so G is F.
  update eq. (2.7) on the whole augmented state, x_0 = (u0, w0, u0, w0) (the
  scheme starts from rest at t = 0); jumps eq. (2.8) on (u, w) through M_H.
k = N sweeps reproduce the uninterrupted scheme exactly.
"""
from __future__ import annotations

import numpy as np

from .parareal import mh_norm
from .scheme import Scheme


def F_carry(sch: Scheme, u, w, ul, wl, F1, F2):
    """P fine steps from (u, w) with lags (ul, wl): (u_P, w_P, u_{P-1}, w_{P-1})."""
    for _ in range(sch.P):
        u1, w1 = sch.step(u, w, ul, wl, sch.dt, F1, F2, sch.cho_f)
        ul, wl, u, w = u, w, u1, w1
    return u, w, ul, wl


def G_carry(sch: Scheme, u, w, ul, wl, F1, F2):
    """One coarse step with the extrapolated lag and the interpolated lag of
    its output."""
    e = sch.Dt / sch.dt
    u1, w1 = sch.step(u, w, u - e * (u - ul), w - e * (w - wl), sch.Dt, F1, F2, sch.cho_G)
    c = sch.dt / sch.Dt
    return u1, w1, u1 - c * (u1 - u), w1 - c * (w1 - w)


def sequential_uninterrupted(sch: Scheme, u0, w0, F1, F2, amp):
    """The scheme over all N P fine steps with the lags carried; returns the
    augmented states at t_0..t_N as arrays [N+1, d] (u, w, u^-, w^-)."""
    u, w, ul, wl = [u0], [w0], [u0], [w0]
    for n in range(sch.N):
        a, b, c, d = F_carry(sch, u[n], w[n], ul[n], wl[n], amp[n] * F1, amp[n] * F2)
        u.append(a)
        w.append(b)
        ul.append(c)
        wl.append(d)
    return np.array(u), np.array(w), np.array(ul), np.array(wl)


def parareal_carry(sch: Scheme, u0, w0, F1, F2, amp, eps, k_max, stats=None):
    """Algorithm 1 on the augmented state with the sequential carrying F;
    returns (u, w, u^-, w^-) at t_0..t_N."""
    red, N = sch.red, sch.N
    F1s = [amp[n] * F1 for n in range(N)]
    F2s = [amp[n] * F2 for n in range(N)]
    X = [(u0, w0, u0, w0)]
    g_old = []
    for n in range(N):                                  # k = 0: G sweep
        g = G_carry(sch, *X[n], F1s[n], F2s[n])
        g_old.append(g)
        X.append(g)
    jumps = []
    k = 0
    for k in range(1, min(k_max, N) + 1):
        Fh = [F_carry(sch, *X[n], F1s[n], F2s[n]) for n in range(N)]
        Xn = [X[0]]
        jump = 0.0
        for n in range(N):
            g = G_carry(sch, *Xn[n], F1s[n], F2s[n])
            x = tuple(g[i] + Fh[n][i] - g_old[n][i] for i in range(4))
            g_old[n] = g
            Xn.append(x)
            jump = max(jump, mh_norm(red, x[0] - X[n + 1][0], x[1] - X[n + 1][1]))
        X = Xn
        jumps.append(jump)
        if jump <= eps:
            break
    if stats is not None:
        stats.update({"K1": k, "jumps": jumps})
    return tuple(np.array([x[i] for x in X]) for i in range(4))
