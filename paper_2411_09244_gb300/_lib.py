"""ctypes binding of libpint.so (declarations in include/pint.h).

Argument marshalling only: arrays may be torch tensors (host or CUDA) or
NumPy arrays; their data pointers are passed through and the library stages
host memory itself.  Loading fails loudly when the shared library is absent:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpint.so")

PINT_OK = 0
STATUS = {0: "OK", -1: "BAD_ARG", -2: "OOM", -3: "CUDA", -4: "UNSTABLE_DT", -5: "NOT_CONVERGED",
          -6: "NONFINITE", -7: "SINGULAR", -8: "STATE", -9: "TIMEOUT"}
PINT_FP64, PINT_MIXED, PINT_MIXED_F32 = 0, 1, 2
PINT_ALLOW_UNSTABLE = 1
PINT_FINE_SEQUENTIAL = 2
PINT_AUTOTUNE = 4
PINT_COARSE_FP64 = 8
PINT_COARSE_GRID = 128
PINT_REFINE_FP64 = 16
PINT_CARRY_LAGS = 32
PINT_ADJOINT_RESPONSE = 64
MAX_ITERS = 512


class SpaceInfo(C.Structure):
    _fields_ = [("n_f", C.c_int), ("nc", C.c_int), ("J", C.c_int), ("ell", C.c_int),
                ("n_blocks", C.c_int), ("n_raw", C.c_int), ("L", C.c_int), ("d1", C.c_int),
                ("d2", C.c_int), ("gamma", C.c_double), ("lambda_max22", C.c_double),
                ("dt_max", C.c_double), ("setup_ms", C.c_double), ("T", C.c_double), ("Dt", C.c_double),
                ("dt", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("K1", C.c_int), ("converged", C.c_int), ("wr_total", C.c_int),
                ("wr_iters", C.c_int * MAX_ITERS), ("jumps", C.c_double * MAX_ITERS),
                ("solve_ms", C.c_double), ("f_ms", C.c_double), ("g_ms", C.c_double),
                ("prolong_ms", C.c_double), ("launches", C.c_int), ("hot_launches", C.c_int),
                ("hot_ms", C.c_double), ("hot_flops", C.c_double)]

    def as_dict(self):
        k = self.K1
        return {"K1": k, "converged": bool(self.converged), "wr_total": self.wr_total,
                "wr_iters": list(self.wr_iters[:k]), "jumps": list(self.jumps[:k]),
                "solve_ms": self.solve_ms, "f_ms": self.f_ms, "g_ms": self.g_ms,
                "prolong_ms": self.prolong_ms, "launches": self.launches,
                "hot_launches": self.hot_launches, "hot_ms": self.hot_ms, "hot_flops": self.hot_flops}


class BatchItem(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("u0_nodes", C.c_void_p), ("f_shape", C.c_void_p), ("amp", C.c_void_p),
                ("eps", C.c_double), ("k_max", C.c_int), ("wr_tol", C.c_double), ("wr_max", C.c_int),
                ("u_out", C.c_void_p), ("coarse_out", C.c_void_p), ("stats", C.POINTER(Stats)),
                ("status", C.c_int)]


class PintError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

SYMBOLS = {
    "pint_setup_fine_grid": [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p],
    "pint_build_multiscale_spaces": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(SpaceInfo)],
    "pint_assemble_reduced": [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                              C.POINTER(SpaceInfo)],
    "pint_parareal_solve": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                            C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(Stats)],
    "pint_sequential_solve": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "pint_adjoint": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                     C.c_double, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double), C.c_void_p,
                     C.c_void_p],
    "pint_get_reduced": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pint_prolong": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "pint_prolong_noalloc": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "pint_apply_G": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "pint_apply_F": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                     C.c_void_p, C.POINTER(C.c_int)],
    "pint_get_info": [C.c_void_p, C.POINTER(SpaceInfo)],
    "pint_destroy": [C.c_void_p],
    "pint_batch_solve": [C.c_void_p, C.c_int, C.c_int],
    "pint_tuning_count": [],
    "pint_tuning_get": [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)],
    "pint_tuning_set": [C.c_void_p, C.c_void_p, C.c_int],
    "pint_tuning_clear": [],
    "pint_set_wait_limit": [C.c_int],
    "pint_set_sweep_smem": [C.c_int],
}


def lib():
    """Load libpint.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, argt in SYMBOLS.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = C.c_int
        L.pint_last_error.restype = C.c_char_p
        L.pint_last_error.argtypes = []
        _lib = L
    return _lib


def check(status: int, allow=()):
    if status != PINT_OK and status not in allow:
        raise PintError(status, lib().pint_last_error().decode())
    return status


def ptr(x):
    """Data pointer of a torch tensor or NumPy array (None -> NULL); the
    array must be contiguous and of the documented dtype."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def current_stream():
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None
