"""The allocation-free prolongation (pint_prolong_noalloc) against the regular
one (pint_prolong), through the C ABI.

pint_prolong_noalloc exists for callers that cannot call cudaMalloc or any
allocating routine (a host runtime that owns the device allocator, a loop
that must not touch it): its scratch is a fixed device array inside the
library.  The call is stream-ordered and returns without waiting, so each
check synchronises first.  This file is named
so that pytest collects it last; it must pass alone in a fresh process and
after the other tests.  Two calls in a row must each match pint_prolong
(the same kernels run in both, so the tolerance of the prolongation parity
test, 1e-10, is far looser than what is observed)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2411_09244_gb300 import api, _lib  # noqa: E402
from paper_2411_09244_gb300.inputs import config_small  # noqa: E402


def _noalloc(p, coarse_dev, out_dev):
    return p.lib.pint_prolong_noalloc(p.h, C.c_void_p(coarse_dev.data_ptr()), coarse_dev.shape[0],
                                      C.c_void_p(out_dev.data_ptr()))


def test_noalloc_prolong_matches_regular_twice():
    prob = config_small(n_f=24, nc=4, J=3, ell=2, N=3, P=12, channels=3, contrast=1e4, f_kind="gauss")
    p = api.from_problem(prob, device="cuda", T=1e-5)
    d = p.info["d1"] + p.info["d2"]
    rng = np.random.default_rng(21)
    for call in range(2):
        X = torch.tensor(rng.normal(size=(3 + call, d)), dtype=torch.float64, device="cuda")
        ref = p.prolong(X)
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(p, X, out) == 0, p.lib.pint_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-10, (call, err)
    p.close()


def test_noalloc_rejects_oversize_and_host_pointers():
    prob = config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
    p = api.from_problem(prob, device="cuda", T=1e-5)
    d = p.info["d1"] + p.info["d2"]
    big = (1 << 20) // (d + p.info["n_raw"]) + 1
    X = torch.zeros((big, d), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, p.nn), dtype=torch.float64, device="cuda")
    assert _noalloc(p, X, out) == -1
    assert b"exceeds" in p.lib.pint_last_error()
    Xh = np.zeros((1, d))
    assert p.lib.pint_prolong_noalloc(p.h, C.c_void_p(Xh.ctypes.data), 1, C.c_void_p(out.data_ptr())) == -1
    p.close()
