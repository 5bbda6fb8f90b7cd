"""Run the oracle's Algorithm 1 to the end on a benchmark workload and record
its iteration counts (test infrastructure, like the rest of this package).

The CPU baseline of the throughput benchmark times bounded samples of the
oracle's solve (one WR iteration on a few intervals, one coarse sweep, the
prolongation) on the workload's own reduced operators and scales them to a
whole solve with these counts: parareal sweeps K1 and the WR iterations of
every sweep.  A full oracle solve of the 256x256 workload takes about 45
minutes on eight cores, too long for every benchmark run, so it is run once
by this script and the counts are stored beside it.

    python -m oracle.record_counts [c1|c2 ...]

writes oracle/counts_<config>.json.  The tolerances are the benchmark's:
eps = the workload's jump tolerance (absolute), wr_tol = 1e-3 eps, at most
200 WR iterations per sweep, the stable final time of the oracle's spaces.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def counts_path(config: str) -> str:
    return os.path.join(HERE, f"counts_{config}.json")


def load_counts(config: str):
    """The stored counts of `config`, or None when they were never recorded."""
    p = counts_path(config)
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        return json.load(fh)


def record(config: str) -> dict:
    from paper_2411_09244_gb300 import inputs
    from .pipeline import OracleRun
    prob = inputs.CONFIGS[config]()
    t0 = time.perf_counter()
    run = OracleRun(prob)
    setup_s = time.perf_counter() - t0
    eps = prob.eps
    t0 = time.perf_counter()
    _, _, st = run.solve(eps=eps, wr_tol=1e-3 * eps, wr_max=200)
    solve_s = time.perf_counter() - t0
    out = {"config": config, "workload": prob.name, "N": prob.N, "P": prob.P, "T": run.T,
           "d1": run.red.d1, "d2": run.red.d2, "eps": eps, "wr_tol": 1e-3 * eps, "wr_max": 200,
           "K1": st["K1"], "wr_iters": [int(x) for x in st["wr_iters"]],
           "wr_total": int(sum(st["wr_iters"])), "jumps": [float(x) for x in st["jumps"]],
           "oracle_setup_s": setup_s, "oracle_solve_s": solve_s,
           "host_cores": len(os.sched_getaffinity(0))}
    with open(counts_path(config), "w") as fh:
        json.dump(out, fh, indent=1)
    return out


if __name__ == "__main__":
    for cfg in (sys.argv[1:] or ["c1", "c2"]):
        print(json.dumps(record(cfg)))
