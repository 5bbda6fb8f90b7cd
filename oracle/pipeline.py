"""Convenience composition of the oracle's stages for one Problem."""
from __future__ import annotations

import time

import numpy as np

from .fem import FineProblem
from .spaces import Spaces
from .reduced import Reduced, stable_T
from .scheme import Scheme
from . import parareal as pr


class OracleRun:
    def __init__(self, prob, T=None):
        t0 = time.perf_counter()
        self.prob = prob
        self.fp = FineProblem(prob.n_f, prob.kappa, prob.nc)
        self.spc = Spaces(self.fp, prob.J, prob.ell)
        self.red = Reduced(self.fp, self.spc)
        self.gamma = self.red.gamma()
        self.lam22 = self.red.lambda_max_22()
        if T is None:
            T = prob.T if prob.T is not None else stable_T(prob.N, self.gamma, self.lam22)
        self.T = T
        self.sch = Scheme(self.red, T, prob.N, prob.P, prob.alpha)
        self.F1, self.F2 = self.red.load(prob.f)
        self.u0, self.w0 = self.red.project_initial(prob.u0)
        self.setup_s = time.perf_counter() - t0

    def solve(self, eps=None, k_max=None, wr_tol=None, wr_max=200, fine="wr"):
        p = self.prob
        eps = p.eps if eps is None else eps
        k_max = p.N if k_max is None else k_max
        wr_tol = 1e-3 * eps if wr_tol is None else wr_tol
        st = {}
        u, w = pr.parareal(self.sch, self.u0, self.w0, self.F1, self.F2, p.amp, eps, k_max,
                           wr_tol, wr_max, fine=fine, stats=st)
        return u, w, st

    def sequential(self):
        p = self.prob
        return pr.sequential_fine(self.sch, self.u0, self.w0, self.F1, self.F2, p.amp)

    def fine_field(self, u, w):
        """[N+1, (n_f+1)^2] prolonged fields."""
        return np.stack([self.red.prolong(u[n], w[n]) for n in range(u.shape[0])])
