"""The autotuner's process-wide table through the C ABI (host-only calls:
no GPU computation).  The measurement itself runs in the mixed-path GPU
tests (PINT_AUTOTUNE)."""
import json

import pytest

from paper_2411_09244_gb300 import api, _lib


@pytest.fixture(autouse=True)
def empty_table():
    from paper_2411_09244_gb300 import build
    import os
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    api.clear_tuning()
    yield
    api.clear_tuning()


ROW = dict(M=1343, Kp=576, ncols=4096, maxs=1, tn=192, s=1, pair=0, us=41.5)


def test_set_get_roundtrip_and_key_order():
    rows = [dict(ROW), dict(ROW, M=257, Kp=2688, maxs=4, tn=256, s=3, us=0.0), dict(ROW, ncols=2048, tn=128, pair=1)]
    api.set_tuning(rows)
    got = api.tuning_table()
    assert len(got) == 3 and _lib.lib().pint_tuning_count() == 3
    keys = [(r["M"], r["Kp"], r["ncols"], r["maxs"]) for r in got]
    assert keys == sorted(keys)
    assert {tuple(sorted(r.items())) for r in got} == {tuple(sorted(r.items())) for r in rows}
    # merging replaces the choice for an existing shape
    api.set_tuning([dict(ROW, tn=224, us=39.0)])
    got = {(r["M"], r["ncols"]): r for r in api.tuning_table()}
    assert got[(1343, 4096)]["tn"] == 224 and len(got) == 3


@pytest.mark.parametrize("bad", [dict(tn=96), dict(tn=288), dict(tn=200), dict(s=0), dict(s=2),
                                 dict(maxs=4, s=3, Kp=584), dict(M=0), dict(ncols=-1), dict(pair=2),
                                 dict(pair=-1)])
def test_invalid_rows_are_rejected_atomically(bad):
    with pytest.raises(_lib.PintError) as ei:
        api.set_tuning([dict(ROW, M=64), dict(ROW, **bad)])
    assert ei.value.status == -1 and "row 1" in str(ei.value)
    assert api.tuning_table() == []


def test_bad_pointer_arguments():
    import ctypes as C
    n = C.c_int(0)
    assert _lib.lib().pint_tuning_get(None, None, 1, C.byref(n)) == -1
    assert _lib.lib().pint_tuning_set(None, None, 2) == -1
    assert _lib.lib().pint_tuning_set(None, None, 0) == 0


def test_json_save_load(tmp_path):
    api.set_tuning([ROW])
    path = tmp_path / "tune.json"
    api.save_tuning(str(path), device="GB300-test")
    doc = json.loads(path.read_text())
    assert doc["version"] == 2 and doc["device"] == "GB300-test" and len(doc["entries"]) == 1
    api.clear_tuning()
    assert api.load_tuning(str(path), device="another") == 0 and api.tuning_table() == []
    assert api.load_tuning(str(path), device="GB300-test") == 1
    assert api.tuning_table()[0]["tn"] == 192
    # a version-1 table (rows without the pairing column) loads as unpaired
    api.clear_tuning()
    old = {k: v for k, v in ROW.items() if k != "pair"}
    path.write_text(json.dumps({"version": 1, "device": "GB300-test", "entries": [old]}))
    assert api.load_tuning(str(path), device="GB300-test") == 1
    assert api.tuning_table()[0]["pair"] == 0


@pytest.mark.gpu
def test_autotuned_mixed_solve():
    """PINT_AUTOTUNE: the first mixed solve times each contraction shape and
    fills the table (one row per shape met, keyed by d1 / d2); the result
    stays within 1e-6 of the FP64 path, and a forced choice from the table
    (every valid tile width, unpaired and in cluster pairs sharing B tiles)
    gives the same answer; pairing changes only which CTA loads which bytes,
    so paired and unpaired solves agree bit for bit."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2411_09244_gb300.inputs import config_small
    prob = config_small(n_f=48, nc=6, J=3, ell=2, N=6, P=32, channels=4, contrast=1e4, f_kind="gauss")
    p = api.from_problem(prob)
    try:
        T = p.T
        _, f64, _ = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-11)
        p.assemble_reduced(T, prob.N, prob.P, prob.alpha, _lib.PINT_MIXED, autotune=True)
        _, fm, st = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-11)
        tab = api.tuning_table()
        d1, d2 = p.info["d1"], p.info["d2"]
        assert tab and {r["M"] for r in tab} <= {d1, d2} and all(r["us"] > 0 for r in tab)
        ref = f64.cpu().numpy()
        err = np.linalg.norm(fm.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 1e-6, err
        for tn in (128, 160, 192, 224, 256):
            got = []
            for pair in (0, 1):
                api.set_tuning([dict(r, tn=tn, s=1, pair=pair) for r in tab])
                _, ft, _ = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=1e-11)
                e = np.linalg.norm(ft.cpu().numpy() - ref) / np.linalg.norm(ref)
                assert e < 1e-6, (tn, pair, e)
                got.append(ft.cpu().numpy())
            assert np.array_equal(got[0], got[1]), tn
    finally:
        p.close()
