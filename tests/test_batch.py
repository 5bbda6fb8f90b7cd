"""The many-instance workload: its seeded recipe (CPU), pint_batch_solve's
argument checks (CPU, no device work), and the batch solve of several
independent instances, each on its own context and CUDA stream, driven by the
library's worker threads (GPU): batch results equal the one-at-a-time results
and the oracle's."""
import numpy as np
import pytest

from paper_2411_09244_gb300.inputs import config_c4

SIZES = (32, 96)  # two coupling shapes: the per-shape kernels of both run in one process


def test_recipe_is_deterministic_and_in_range():
    seen = set()
    for i in range(48):
        a, b = config_c4(i), config_c4(i)
        assert a.n_f == b.n_f and a.J == b.J and a.N == b.N
        assert np.array_equal(a.kappa, b.kappa) and np.array_equal(a.f, b.f)
        assert a.n_f in (64, 96, 128, 192, 256)
        assert a.nc * 8 == a.n_f
        assert 2 <= a.J <= 4 and a.ell == 2 and a.P == 32 and a.N in (16, 32, 64)
        c = a.meta["contrast"]
        assert 1e3 <= c <= 1e6
        assert 5 <= a.meta["channels"] <= 50 and 5 <= a.meta["inclusions"] <= 50
        assert a.kappa.size == a.n_f * a.n_f
        assert a.kappa.min() == 1.0 and np.isclose(a.kappa.max(), c)
        assert a.u0.shape == ((a.n_f + 1) ** 2,) and not a.u0.any()
        assert np.array_equal(a.amp, np.ones(a.N))
        seen.add((a.n_f, a.N))
    # uneven: the draws span several sizes and interval counts
    assert len({s for s, _ in seen}) >= 4 and len({n for _, n in seen}) == 3
    assert not np.array_equal(config_c4(0).f[:64], config_c4(1).f[:64])


def test_recipe_honours_sizes():
    got = {config_c4(i, sizes=SIZES).n_f for i in range(4)}
    assert got == set(SIZES)


def test_batch_arguments_are_checked_without_gpu():
    import ctypes as C
    from paper_2411_09244_gb300 import _lib
    L = _lib.lib()
    assert L.pint_batch_solve(None, 0, 0) == 0
    assert L.pint_batch_solve(None, 2, 0) == -1
    items = (_lib.BatchItem * 2)()
    assert L.pint_batch_solve(C.cast(items, C.c_void_p), 2, 0) == -1          # NULL contexts
    assert b"item 0" in L.pint_last_error()
    items[0].ctx = items[1].ctx = 0x1000                                       # repeated context
    assert L.pint_batch_solve(C.cast(items, C.c_void_p), 2, 0) == -1
    assert b"item 1" in L.pint_last_error()


@pytest.mark.gpu
def test_batch_equals_sequential_and_oracle():
    torch = pytest.importorskip("torch")
    from paper_2411_09244_gb300 import api
    from paper_2411_09244_gb300._lib import PINT_MIXED, PINT_FP64
    from oracle.pipeline import OracleRun
    probs = [config_c4(i, sizes=SIZES) for i in range(4)]   # relative eps (see config_c4)
    pints = []
    try:
        for prob in probs:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                p = api.Pint(prob.n_f, prob.kappa)
                p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
                p.assemble_reduced(None, prob.N, prob.P, prob.alpha)
            pints.append(p)
        torch.cuda.synchronize()
        seq = []
        for p, prob in zip(pints, probs):
            with torch.cuda.stream(p.stream):
                seq.append(p.parareal_solve(prob.u0, prob.f, prob.amp, eps=prob.eps))
            p.stream.synchronize()
        con = api.solve_batch(pints, probs, want_fine=True)
        # the reductions use atomics, so the two runs agree to rounding, not bitwise
        for (cs, fs, ss), (cc, fc, sc) in zip(seq, con):
            assert ss["K1"] == sc["K1"]
            assert float(torch.linalg.norm(cc - cs) / torch.linalg.norm(cs)) < 1e-11
            assert float(torch.linalg.norm(fc - fs) / torch.linalg.norm(fs)) < 1e-11
        # the first instance: the GPU's sequential fine scheme against the
        # oracle's (FP64 bar 1e-10), and the parareal result (jump tolerance
        # 1e-10) against that sequential solution
        orc = OracleRun(probs[0], T=pints[0].T)
        u, w = orc.sequential()
        ref = orc.fine_field(u, w)[1:]
        with torch.cuda.stream(pints[0].stream):
            _, f_seq = pints[0].sequential_solve(probs[0].u0, probs[0].f, probs[0].amp)
        pints[0].stream.synchronize()
        f_seq = f_seq.cpu().numpy()
        assert np.linalg.norm(f_seq - ref) / np.linalg.norm(ref) < 1e-10
        got = con[0][1].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-7
        # mixed precision, concurrently, within 1e-6 of the FP64 results (L2
        # over the whole trajectory: the solver's tolerances are relative to
        # the largest state, and with u0 = 0 the first states are ~1e-5 of it)
        for p, prob in zip(pints, probs):
            with torch.cuda.stream(p.stream):
                p.assemble_reduced(p.T, prob.N, prob.P, prob.alpha, PINT_MIXED)
        torch.cuda.synchronize()
        mix = api.solve_batch(pints, probs, want_fine=True)
        for (_, fs, _), (_, fm, _) in zip(seq, mix):
            assert float(torch.linalg.norm(fm - fs) / torch.linalg.norm(fs)) < 1e-6
        for p, prob in zip(pints, probs):
            with torch.cuda.stream(p.stream):
                p.assemble_reduced(p.T, prob.N, prob.P, prob.alpha, PINT_FP64)
    finally:
        for p in pints:
            p.close()


@pytest.mark.gpu
def test_batch_reports_the_failing_item():
    """An item whose context has no time grid fails with STATE; the others are
    solved, and the call returns the failing item's status and index."""
    torch = pytest.importorskip("torch")
    from paper_2411_09244_gb300 import api, _lib
    probs = [config_c4(i, sizes=(32,)) for i in range(2)]
    pints = []
    try:
        for k, prob in enumerate(probs):
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                p = api.Pint(prob.n_f, prob.kappa)
                p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
                if k == 0:
                    p.assemble_reduced(None, prob.N, prob.P, prob.alpha)
                else:  # no time grid yet: N, P and d for the outputs taken from the first
                    p.info = dict(pints[0].info)
                    p.N, p.P = probs[0].N, probs[0].P
            pints.append(p)
        probs[1].amp = probs[0].amp
        plan = api.BatchPlan(pints, probs)
        with pytest.raises(_lib.PintError, match="STATE") as ei:
            plan.run()
        assert "item 1" in str(ei.value)
        assert plan.items[0].status == 0 and plan.items[1].status == -8
    finally:
        for p in pints:
            p.close()
