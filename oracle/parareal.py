"""Algorithm 1: parareal all-at-once partially explicit splitting.

Reading of the garbled indices of Algorithm 1 (it applies F to u^{k-1} but
updates with G(u^k)): the standard update eq. (2.7),
  x_{n+1}^{k} = G(x_n^{k}) + F(x_n^{k-1}) - G(x_n^{k-1}),  x_0^k = x_0,
where x = (u, w) is the V_H1 x V_H2 state; k = 0 is the initial G sweep and
k counts F sweeps.  Stopping rule eq. (2.8) on the combined V_H function,
max_{1<=n<=N} ||(u+w)_n^k - (u+w)_n^{k-1}||_{L2} <= eps (absolute), the L2
norm taken through M_H; the loop also ends at k = N (the sweep is then exact)
or at k_max.

The fine propagator is the WR solver of scheme.Scheme.F_wr, or the
sequential fine scheme when `fine="seq"`.
"""
from __future__ import annotations

import numpy as np

from .scheme import Scheme


def mh_norm(red, du, dw):
    v = red.M11 @ du
    s = du @ v + 2.0 * du @ (red.M12 @ dw) + dw @ (red.M22 @ dw)
    return float(np.sqrt(max(s, 0.0)))


def parareal(sch: Scheme, u0, w0, F1, F2, amp, eps, k_max, wr_tol, wr_max, fine="wr",
             stats=None):
    """Returns the coarse states X[k_final] as arrays u[N+1, d1], w[N+1, d2]."""
    red = sch.red
    N = sch.N
    F1s = [amp[n] * F1 for n in range(N)]
    F2s = [amp[n] * F2 for n in range(N)]
    u = [u0]
    w = [w0]
    g_old = []
    for n in range(N):                                  # k = 0: G sweep
        un, wn = sch.G(u[n], w[n], F1s[n], F2s[n])
        g_old.append((un, wn))
        u.append(un)
        w.append(wn)
    jumps, wr_iters = [], []
    k = 0
    for k in range(1, min(k_max, N) + 1):
        starts = [(u[n], w[n]) for n in range(N)]
        if fine == "wr":
            Fh, it = sch.F_wr(starts, F1s, F2s, wr_tol, wr_max)
        else:
            Fh = [sch.F_seq(s[0], s[1], F1s[n], F2s[n]) for n, s in enumerate(starts)]
            it = 0
        wr_iters.append(it)
        un_new = [u0]
        wn_new = [w0]
        jump = 0.0
        for n in range(N):
            gu, gw = sch.G(un_new[n], wn_new[n], F1s[n], F2s[n])
            nu = gu + Fh[n][0] - g_old[n][0]
            nw = gw + Fh[n][1] - g_old[n][1]
            g_old[n] = (gu, gw)
            un_new.append(nu)
            wn_new.append(nw)
            jump = max(jump, mh_norm(red, nu - u[n + 1], nw - w[n + 1]))
        u, w = un_new, wn_new
        jumps.append(jump)
        if jump <= eps:
            break
    if stats is not None:
        stats.update({"K1": k, "jumps": jumps, "wr_iters": wr_iters})
    return np.array(u), np.array(w)


def sequential_fine(sch: Scheme, u0, w0, F1, F2, amp):
    """u_h^*: the fine scheme run interval after interval (restart lags at
    each coarse boundary), the limit of Algorithm 1."""
    u = [u0]
    w = [w0]
    for n in range(sch.N):
        un, wn = sch.F_seq(u[n], w[n], amp[n] * F1, amp[n] * F2)
        u.append(un)
        w.append(wn)
    return np.array(u), np.array(w)
