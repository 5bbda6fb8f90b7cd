"""Python front end of libpint with the C-ABI names (include/pint.h).

`Pint` owns one context.  Inputs may be NumPy arrays, host tensors or CUDA
tensors (float64, contiguous); results come back as float64 tensors on the
device the caller asks for.  Every numerical step runs in libpint's CUDA
kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _f64(x, device=None):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(dtype=torch.float64)
    if device is not None:
        x = x.to(device)
    return x.contiguous()


class Pint:
    """One problem instance: fine grid -> spaces -> reduced operators ->
    solves.  Mirrors pint_setup_fine_grid / pint_build_multiscale_spaces /
    pint_assemble_reduced / pint_parareal_solve / pint_adjoint."""

    def __init__(self, n_f: int, kappa_cells, device: str = "cuda"):
        self.device = torch.device(device)
        self.lib = L.lib()
        self.n_f = n_f
        self.nn = (n_f + 1) ** 2
        k = _f64(kappa_cells, self.device).reshape(-1)
        h = C.c_void_p()
        self.stream = torch.cuda.current_stream(self.device) if torch.cuda.is_available() else None
        L.check(self.lib.pint_setup_fine_grid(C.byref(h), n_f, L.ptr(k), L.current_stream()))
        self.h = h
        self.info = None

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.pint_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stages -----------------------------------------------------------
    def build_multiscale_spaces(self, nc: int, J: int, ell: int) -> dict:
        info = L.SpaceInfo()
        L.check(self.lib.pint_build_multiscale_spaces(self.h, nc, J, ell, C.byref(info)))
        self.info = info.as_dict()
        return self.info

    def assemble_reduced(self, T: float | None, N: int, P: int, alpha: float, precision: int = L.PINT_FP64,
                         allow_unstable: bool = False, fine_sequential: bool = False,
                         autotune: bool = False, coarse_fp64: bool = False, refine_fp64: bool = False,
                         carry_lags: bool = False, adjoint_response: bool = False,
                         coarse_grid: bool = False) -> dict:
        """T = None (passed as 0) lets the library pick the stable final time
        of Section 3.2; the T used is returned in info["T"].
        fine_sequential: PINT_FINE_SEQUENTIAL (FP64 path comparison mode).
        autotune: PINT_AUTOTUNE (measured contraction tiles, mixed path).
        coarse_fp64: PINT_COARSE_FP64 (every coarse sweep of the mixed path in FP64).
        refine_fp64: PINT_REFINE_FP64 (refinement residual contractions in FP64).
        carry_lags: PINT_CARRY_LAGS (lag-carrying comparison variant, FP64).
        adjoint_response: PINT_ADJOINT_RESPONSE (amplitude gradient by <lambda_{n+1}, s>).
        coarse_grid: PINT_COARSE_GRID (the first solve's FP32 coarse sweeps grid-wide)."""
        info = L.SpaceInfo()
        flags = ((L.PINT_ALLOW_UNSTABLE if allow_unstable else 0) | (L.PINT_FINE_SEQUENTIAL if fine_sequential else 0)
                 | (L.PINT_AUTOTUNE if autotune else 0) | (L.PINT_COARSE_FP64 if coarse_fp64 else 0)
                 | (L.PINT_REFINE_FP64 if refine_fp64 else 0) | (L.PINT_CARRY_LAGS if carry_lags else 0)
                 | (L.PINT_ADJOINT_RESPONSE if adjoint_response else 0) | (L.PINT_COARSE_GRID if coarse_grid else 0))
        st = self.lib.pint_assemble_reduced(self.h, 0.0 if T is None else T, N, P, alpha, precision, flags,
                                            C.byref(info))
        L.check(st)
        self.info = info.as_dict()
        self.T, self.N, self.P, self.alpha = info.T, N, P, alpha
        return self.info

    def get_info(self) -> dict:
        info = L.SpaceInfo()
        L.check(self.lib.pint_get_info(self.h, C.byref(info)))
        return info.as_dict()

    # -- solves -----------------------------------------------------------
    def parareal_solve(self, u0_nodes, f_shape, amp=None, eps=1e-10, k_max=None, wr_tol=None, wr_max=200,
                       want_fine=True, out_device=None):
        dev = self.device if out_device is None else torch.device(out_device)
        u0 = _f64(u0_nodes, self.device)
        f = _f64(f_shape, self.device)
        a = _f64(amp, self.device)
        k_max = self.N if k_max is None else k_max
        wr_tol = 1e-3 * eps if wr_tol is None else wr_tol
        d = self.info["d1"] + self.info["d2"]
        coarse = torch.empty((self.N + 1, d), dtype=torch.float64, device=dev)
        fine = torch.empty((self.N, self.nn), dtype=torch.float64, device=dev) if want_fine else None
        st = L.Stats()
        status = self.lib.pint_parareal_solve(self.h, L.ptr(u0), L.ptr(f), L.ptr(a), eps, k_max, wr_tol,
                                              wr_max, L.ptr(fine), L.ptr(coarse), C.byref(st))
        L.check(status, allow=(-5,))
        out = st.as_dict()
        out["status"] = L.STATUS[status]
        return coarse, fine, out

    def sequential_solve(self, u0_nodes, f_shape, amp=None, want_fine=True):
        u0 = _f64(u0_nodes, self.device)
        f = _f64(f_shape, self.device)
        a = _f64(amp, self.device)
        d = self.info["d1"] + self.info["d2"]
        coarse = torch.empty((self.N + 1, d), dtype=torch.float64, device=self.device)
        fine = torch.empty((self.N, self.nn), dtype=torch.float64, device=self.device) if want_fine else None
        L.check(self.lib.pint_sequential_solve(self.h, L.ptr(u0), L.ptr(f), L.ptr(a), L.ptr(fine),
                                               L.ptr(coarse)))
        return coarse, fine

    def get_reduced(self, which: str, aux=None):
        names = {"M11": 0, "A11": 1, "M22": 2, "A22": 3, "M12": 4, "A12": 5, "load": 6, "GM": 7, "kinds": 8,
                 "setup_ms": 9}
        d1, d2, nr = self.info["d1"], self.info["d2"], self.info["n_raw"]
        shapes = {"M11": (d1, d1), "A11": (d1, d1), "M22": (d2, d2), "A22": (d2, d2), "M12": (d1, d2),
                  "A12": (d1, d2), "load": (d1 + d2,), "GM": (nr, nr), "kinds": (nr, 2), "setup_ms": (6,)}
        out = torch.empty(shapes[which], dtype=torch.float64, device=self.device)
        x = _f64(aux, self.device)
        L.check(self.lib.pint_get_reduced(self.h, names[which], L.ptr(out), L.ptr(x)))
        return out

    def prolong(self, coarse):
        c = _f64(coarse, self.device)
        cnt = c.shape[0]
        out = torch.empty((cnt, self.nn), dtype=torch.float64, device=self.device)
        L.check(self.lib.pint_prolong(self.h, L.ptr(c), cnt, L.ptr(out)))
        return out

    def apply_G(self, states, f_shape, amp=None):
        s = _f64(states, self.device)
        f = _f64(f_shape, self.device)
        a = _f64(amp, self.device)
        out = torch.empty_like(s)
        L.check(self.lib.pint_apply_G(self.h, L.ptr(s), s.shape[0], L.ptr(f), L.ptr(a), L.ptr(out)))
        return out

    def apply_F(self, states, f_shape, amp=None, wr_tol=1e-14, wr_max=200):
        s = _f64(states, self.device)
        f = _f64(f_shape, self.device)
        a = _f64(amp, self.device)
        out = torch.empty_like(s)
        it = C.c_int(0)
        L.check(self.lib.pint_apply_F(self.h, L.ptr(s), s.shape[0], L.ptr(f), L.ptr(a), wr_tol, wr_max,
                                      L.ptr(out), C.byref(it)))
        return out, it.value


    def adjoint(self, obs_nodes, data, u0_nodes, f_shape, amp=None, eps=1e-10, k_max=None, wr_tol=None,
                wr_max=200):
        """pint_adjoint: (J, dJ/du0 [(n_f+1)^2], dJ/damp [N]) of the misfit
        J = 1/2 sum_{n=1..N} sum_o (u_H^n(x_o) - data[n-1, o])^2."""
        obs = torch.as_tensor(np.asarray(obs_nodes), dtype=torch.int32).contiguous()
        d = _f64(data, self.device)
        u0 = _f64(u0_nodes, self.device)
        f = _f64(f_shape, self.device)
        a = _f64(amp, self.device)
        k_max = self.N if k_max is None else k_max
        wr_tol = 1e-3 * eps if wr_tol is None else wr_tol
        J = C.c_double(0.0)
        g_u0 = torch.empty(self.nn, dtype=torch.float64, device=self.device)
        g_amp = torch.empty(self.N, dtype=torch.float64, device=self.device)
        L.check(self.lib.pint_adjoint(self.h, L.ptr(obs), int(obs.numel()), L.ptr(d), L.ptr(u0), L.ptr(f),
                                      L.ptr(a), eps, k_max, wr_tol, wr_max, C.byref(J), L.ptr(g_u0),
                                      L.ptr(g_amp)))
        return J.value, g_u0, g_amp


class ObservationMisfit(torch.autograd.Function):
    """J(u0, amp) = 1/2 sum_{n,o} (u_H^n(x_o) - d_{o,n})^2 through the limit of
    Algorithm 1; backward runs the adjoint (backward) parareal sweep of
    pint_adjoint.  Usage: J = ObservationMisfit.apply(u0, amp, pint, obs, data, f_shape, opts)."""

    @staticmethod
    def forward(ctx, u0, amp, pint, obs_nodes, data, f_shape, opts=None):
        opts = dict(opts or {})
        J, g_u0, g_amp = pint.adjoint(obs_nodes, data, u0.detach(), f_shape, amp.detach(), **opts)
        ctx.save_for_backward(g_u0.to(u0.device, u0.dtype), g_amp.to(amp.device, amp.dtype))
        return torch.tensor(J, dtype=u0.dtype, device=u0.device)

    @staticmethod
    def backward(ctx, grad_out):
        g_u0, g_amp = ctx.saved_tensors
        return grad_out * g_u0, grad_out * g_amp, None, None, None, None, None


# -- autotuner table ----------------------------------------------------------
TUNING_KEYS = ("M", "Kp", "ncols", "maxs", "tn", "s", "pair")


def tuning_table() -> list[dict]:
    """Rows of the process-wide contraction tuning table (pint_tuning_get)."""
    lb = L.lib()
    n = lb.pint_tuning_count()
    rows = np.zeros((max(n, 1), len(TUNING_KEYS)), dtype=np.int32)
    us = np.zeros(max(n, 1), dtype=np.float32)
    got = C.c_int(0)
    L.check(lb.pint_tuning_get(rows.ctypes.data, us.ctypes.data, n, C.byref(got)))
    return [dict(zip(TUNING_KEYS, map(int, rows[i])), us=float(us[i])) for i in range(got.value)]


def set_tuning(entries) -> None:
    """Merge rows (dicts with TUNING_KEYS, optional "us") into the table."""
    entries = list(entries)
    rows = np.array([[int(e.get(k, 0) if k == "pair" else e[k]) for k in TUNING_KEYS] for e in entries],
                    dtype=np.int32).reshape(-1, len(TUNING_KEYS))
    us = np.array([float(e.get("us", 0.0)) for e in entries], dtype=np.float32)
    L.check(L.lib().pint_tuning_set(rows.ctypes.data if len(entries) else None,
                                    us.ctypes.data if len(entries) else None, len(entries)))


def clear_tuning() -> None:
    L.check(L.lib().pint_tuning_clear())


def save_tuning(path: str, device: str | None = None) -> None:
    """Write the table as JSON: {"version": 2, "device": ..., "entries": [...]}."""
    import json
    if device is None and torch.cuda.is_available():
        device = torch.cuda.get_device_name()
    with open(path, "w") as fh:
        json.dump({"version": 2, "device": device, "entries": tuning_table()}, fh, indent=1)


def load_tuning(path: str, device: str | None = None) -> int:
    """Merge a table written by save_tuning; entries measured on another
    device name are skipped.  Returns the number of rows merged."""
    import json
    with open(path) as fh:
        doc = json.load(fh)
    if doc.get("version") not in (1, 2):  # version 1 rows have no "pair" (unpaired)
        raise ValueError(f"{path}: unknown tuning table version {doc.get('version')!r}")
    if device is None and torch.cuda.is_available():
        device = torch.cuda.get_device_name()
    if device is not None and doc.get("device") not in (None, device):
        return 0
    set_tuning(doc["entries"])
    return len(doc["entries"])


class BatchPlan:
    """Prepared arguments of pint_batch_solve for a list of Pints and their
    problems: inputs and output buffers are allocated once (on the device,
    or pinned on the host with host=True, where the library stages the
    copies), so repeated runs allocate nothing."""

    def __init__(self, pints, problems, eps=None, wr_max=200, want_fine=False, host=False):
        self.n = len(pints)
        self.items = (L.BatchItem * max(self.n, 1))()
        self.keep, self.outs = [], []

        def buf(shape, p):
            if host:
                return torch.empty(shape, dtype=torch.float64).pin_memory()
            return torch.empty(shape, dtype=torch.float64, device=p.device)

        for i, (p, prob) in enumerate(zip(pints, problems)):
            if host:
                u0, f, a = (torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
                            for x in (prob.u0, prob.f, prob.amp))
            else:
                u0, f, a = _f64(prob.u0, p.device), _f64(prob.f, p.device), _f64(prob.amp, p.device)
            e = prob.eps if eps is None else eps
            d = p.info["d1"] + p.info["d2"]
            coarse = buf((p.N + 1, d), p)
            fine = buf((p.N, p.nn), p) if want_fine else None
            st = L.Stats()
            self.keep += [u0, f, a]
            it = self.items[i]
            it.ctx = p.h.value
            it.u0_nodes, it.f_shape, it.amp = L.ptr(u0), L.ptr(f), L.ptr(a)
            it.eps, it.k_max, it.wr_tol, it.wr_max = e, p.N, 1e-3 * e, wr_max
            it.u_out, it.coarse_out = L.ptr(fine), L.ptr(coarse)
            it.stats = C.pointer(st)
            self.outs.append((coarse, fine, st))
        self.h2d_bytes = sum(x.numel() * 8 for x in self.keep) if host else 0
        self.d2h_bytes = sum(c.numel() * 8 + (f.numel() * 8 if f is not None else 0)
                             for c, f, _ in self.outs) if host else 0

    def run(self, workers=0):
        """pint_batch_solve over the plan; returns [(coarse, fine, stats)]."""
        if torch.cuda.is_available():
            torch.cuda.synchronize()     # inputs staged on the caller's stream are complete
        status = L.lib().pint_batch_solve(C.cast(self.items, C.c_void_p), self.n, workers)
        L.check(status, allow=(-5,))
        res = []
        for i, (coarse, fine, st) in enumerate(self.outs):
            dct = st.as_dict()
            dct["status"] = L.STATUS[self.items[i].status]
            res.append((coarse, fine, dct))
        return res


def solve_batch(pints, problems, eps=None, wr_max=200, want_fine=False, workers=0, host=False):
    """Solve several independent instances at once through pint_batch_solve:
    the library drives each Pint's context on its own CUDA stream (the
    stream the Pint was created on) from its own worker threads, longest
    instance first, so the GPU overlaps the instances' kernels.  Returns
    [(coarse, fine or None, stats)] in the order of `pints`."""
    return BatchPlan(pints, problems, eps, wr_max, want_fine, host).run(workers)


def from_problem(prob, device="cuda", precision=L.PINT_FP64, T=None):
    """Build a Pint for a seeded Problem (inputs module) through all setup stages."""
    p = Pint(prob.n_f, prob.kappa, device=device)
    p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
    p.assemble_reduced(T if T is not None else prob.T, prob.N, prob.P, prob.alpha, precision)
    return p
