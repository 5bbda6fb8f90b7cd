"""Throughput of the parareal all-at-once partially explicit splitting solve.

One step = one pint_parareal_solve on the 256x256 / 16x16-coarse / J=4 /
four-layer workload with N = 64 coarse intervals x P = 64 fine steps
(initial G sweep, K1 parareal iterations of WR fine propagation on all
intervals + sequential coarse correction + jump norm, prolongation of the N
states to the fine grid), inputs resident in HBM.

metric: DOF.steps/s = (n_f - 1)^2 interior fine unknowns x N P fine steps /
solve time.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the oracle (CPU baseline, reference arm) uses every host core the process may run on
_CORES = len(os.sched_getaffinity(0))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF·steps/s of parareal solve at rel L2 err ≤1e-6 vs FP64; % roofline; iters"
UNIT = "DOF*steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="contraction tiles from the cost model instead of measured (mixed path)")
    ap.add_argument("--tuning", default=None,
                    help="JSON tuning table: loaded before the run if present, written after it")
    ap.add_argument("--batch", type=int, default=16, help="instances of the many-instance workload (c4)")
    ap.add_argument("--workers", type=int, default=0,
                    help="host worker threads of the many-instance batch (0: min(instances, 16))")
    ap.add_argument("--batch-sizes", default="64,96,128",
                    help="fine grid sizes drawn for the c4 instances (comma separated)")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--coarse-fp64", action="store_true",
                    help="mixed path: the low-precision solve's coarse sweeps in FP64 too (PINT_COARSE_FP64)")
    ap.add_argument("--refine-fp64", action="store_true",
                    help="mixed path: refinement residual contractions in FP64 (PINT_REFINE_FP64)")
    return ap.parse_args()


def dist_init(args=None):
    """Ranks from the torchrun environment; NCCL on GPUs, gloo without (tests)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_instances(rank, batch):
    """Seeded instances of one rank in the many-instance run: disjoint blocks per
    rank (weak scaling, no exchange between ranks)."""
    return [rank * batch + i for i in range(batch)]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 DGEMM throughput measured on this machine's GB300 with cuBLAS (torch.matmul
# float64, 4096^3, best of 10); MEASURED_PEAKS.json carries no FP64 figure.
FP64_MEASURED_TFLOPS = 1.096

# DRAM bytes (read + write) per launch of the tensor-core contraction on this
# workload, averaged over its two launches, from the ncu capture summarised in
# profiles/k_wr_umma_c2_mixed.md; only valid for the kernel source it was taken on.
UMMA_TRAFFIC = {"sha1": "c3188baec9826fb3cf93327189aa758ee4297bd4",
                "bytes": (25.104384e6 + 0.021504e6 + 93.655040e6 + 2.986240e6) / 2}


def umma_traffic():
    import hashlib
    path = os.path.join(ROOT, "paper_2411_09244_gb300", "csrc", "k_umma.cu")
    try:
        with open(path, "rb") as fh:
            h = hashlib.sha1(fh.read()).hexdigest()
    except OSError:
        return None
    return UMMA_TRAFFIC["bytes"] if h == UMMA_TRAFFIC["sha1"] else None


def workload_desc(prob):
    return (f"{prob.name}: {prob.n_f}x{prob.n_f} fine, {prob.nc}x{prob.nc} coarse, J={prob.J}, "
            f"ell={prob.ell}, N={prob.N} x P={prob.P}")


def mixed_dtype(args):
    """Arithmetic of the timed solve: the fine propagator's products and the
    rest of the low-precision solve, then what runs in FP64 or double-float."""
    if args.precision == "fp64":
        return "f64"
    lo = "tf32x3/f32" if args.precision == "mixed" else "f32"
    ref = "f64" if getattr(args, "refine_fp64", False) else "double-float (f32 pairs)"
    return f"{lo}; f64 jumps, states and correction coarse step; {ref} refinement residual"


def problem(name):
    from paper_2411_09244_gb300 import inputs
    return {"c1": inputs.config_c1, "c2": inputs.config_c2, "c5": inputs.config_c5}[name]()


class OracleSampler:
    """The oracle as it stands, timed on the host cores on the workload's own
    operators.  Setup (the oracle's multiscale spaces and reduced matrices,
    its time-grid factorisations) is done once and reported, not counted: the
    GPU figure excludes setup too.  A sample times the units of the oracle's
    solve: one WR iteration of the fine propagator on `nsub` intervals, one
    coarse sweep over all N intervals, the prolongation of one state; a whole
    solve is then  sum K0 x N x t_wr + (K1 + 1) x t_G + N x t_prolong,  with
    K1 and the WR iterations of every sweep taken from a complete oracle
    solve of the same workload (oracle/counts_<config>.json, written by
    oracle/record_counts.py).  The 64x64 workload is small enough to time
    whole solves instead."""

    def __init__(self, config, prob):
        from oracle.pipeline import OracleRun
        from oracle.record_counts import load_counts
        self.config, self.prob = config, prob
        self.counts = load_counts(config)
        t0 = time.perf_counter()
        self.run = OracleRun(prob)
        self.setup_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.run.sch._shift_lu()          # the factorisations of eq. (4.7), once per time grid
        self.grid_s = time.perf_counter() - t0
        self.cores = int(os.environ.get("OPENBLAS_NUM_THREADS", _CORES))
        self.D = (prob.n_f - 1) ** 2

    def full_solve(self):
        """One complete oracle solve (64x64 workload): seconds and stats."""
        p = self.prob
        t0 = time.perf_counter()
        u, w, st = self.run.solve(eps=p.eps, wr_tol=1e-3 * p.eps, wr_max=200)
        self.run.fine_field(u[1:], w[1:])
        return time.perf_counter() - t0, st

    def units(self, nsub):
        """(t_wr per interval, t_G per sweep, t_prolong per state), timed now."""
        run, p = self.run, self.prob
        N, nsub = p.N, max(1, min(nsub, p.N))
        starts = [(run.u0, run.w0)] * nsub
        t0 = time.perf_counter()
        run.sch.F_wr(starts, [run.F1] * nsub, [run.F2] * nsub, wr_tol=0.0, wr_max=1)
        t_wr = (time.perf_counter() - t0) / nsub
        t0 = time.perf_counter()
        u, w = run.u0, run.w0
        for n in range(N):
            u, w = run.sch.G(u, w, p.amp[n] * run.F1, p.amp[n] * run.F2)
        t_g = time.perf_counter() - t0
        t0 = time.perf_counter()
        run.red.prolong(u, w)
        t_pr = time.perf_counter() - t0
        return t_wr, t_g, t_pr

    def sample(self, nsub):
        """Seconds per solve extrapolated from one timed sample, and its description."""
        c = self.counts
        if c is None:
            raise RuntimeError(f"oracle/counts_{self.config}.json is missing: run "
                               f"`python -m oracle.record_counts {self.config}`")
        p = self.prob
        t_wr, t_g, t_pr = self.units(nsub)
        t = c["wr_total"] * p.N * t_wr + (c["K1"] + 1) * t_g + p.N * t_pr
        desc = (f"oracle on the workload's own reduced system (d1={self.run.red.d1}, d2={self.run.red.d2}, "
                f"N={p.N}, P={p.P}), {self.cores} threads; measured: one WR iteration on {min(nsub, p.N)} of "
                f"{p.N} intervals ({t_wr:.3f} s per interval), one coarse sweep ({t_g:.3f} s), one "
                f"prolongation ({t_pr:.3f} s); scaled to a solve with the counts of a complete oracle solve "
                f"(K1={c['K1']}, sum K0={c['wr_total']}): {t:.1f} s; setup excluded (spaces "
                f"{self.setup_s:.1f} s, eq. (4.7) factorisations {self.grid_s:.1f} s)")
        return t, desc


def cpu_baseline(config, prob, budget_s=20.0):
    """cpu_baseline of the bench line: the oracle on the host cores."""
    smp = OracleSampler(config, prob)
    out = {"unit": UNIT, "cores": smp.cores, "kind": "oracle"}
    if config == "c1":
        t, st = smp.full_solve()
        out.update(value=smp.D * prob.N * prob.P / t,
                   sample=f"one complete oracle solve of the workload ({t:.2f} s, K1={st['K1']}, "
                          f"sum K0={sum(st['wr_iters'])}), {smp.cores} threads, setup excluded "
                          f"({smp.setup_s:.1f} s)")
        return out
    t1, _, _ = smp.units(1)
    nsub = int(max(1, min(prob.N, budget_s / max(t1, 1e-3) / 2)))
    t, desc = smp.sample(nsub)
    out.update(value=smp.D * prob.N * prob.P / t, sample=desc, oracle_setup_s=smp.setup_s)
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2411_09244_gb300 import api, _lib
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = problem(args.config)
    prec = {"fp64": _lib.PINT_FP64, "mixed": _lib.PINT_MIXED, "mixed_f32": _lib.PINT_MIXED_F32}[args.precision]
    t0 = time.perf_counter()
    p = api.Pint(prob.n_f, prob.kappa, device=dev)
    info = p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
    info = p.assemble_reduced(None, prob.N, prob.P, prob.alpha, _lib.PINT_FP64)
    setup_s = time.perf_counter() - t0
    stages = [round(float(x) / 1e3, 3) for x in p.get_reduced("setup_ms").cpu().tolist()]
    u0 = torch.tensor(prob.u0, dtype=torch.float64, device=dev)
    f = torch.tensor(prob.f, dtype=torch.float64, device=dev)
    amp = torch.tensor(prob.amp, dtype=torch.float64, device=dev)
    eps = prob.eps
    # FP64 GPU path: accuracy reference and the comparison figure
    _, fine64, st64 = p.parareal_solve(u0, f, amp, eps=eps, want_fine=True)
    torch.cuda.synchronize()
    if prec != _lib.PINT_FP64:
        info = p.assemble_reduced(p.T, prob.N, prob.P, prob.alpha, prec, autotune=not args.no_autotune,
                                  coarse_fp64=args.coarse_fp64, refine_fp64=args.refine_fp64)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        p.parareal_solve(u0, f, amp, eps=eps, want_fine=True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times, stats = [], []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush between timed iterations
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("solve")
            e0.record(stream)
            _, fine, st = p.parareal_solve(u0, f, amp, eps=eps, want_fine=True)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            stats.append(st)
    bad = [s["status"] for s in stats if s["status"] != "OK" or not s["converged"]]
    if bad:
        raise SystemExit(f"bench: {len(bad)} timed solves did not converge ({bad[0]}); no number reported")
    rel_err = max(float(torch.linalg.norm(fine[n] - fine64[n]) / torch.linalg.norm(fine64[n]))
                  for n in range(prob.N) if float(torch.linalg.norm(fine64[n])) > 0)
    torch.cuda.synchronize()
    barrier(world)
    t_step = max_over_ranks(sum(times) / len(times), world)
    D = (prob.n_f - 1) ** 2
    dofsteps = D * prob.N * prob.P
    value = world * dofsteps / t_step
    # end to end through the C ABI with pinned host buffers (copies inside)
    hu0 = torch.tensor(prob.u0, dtype=torch.float64).pin_memory()
    hf = torch.tensor(prob.f, dtype=torch.float64).pin_memory()
    ha = torch.tensor(prob.amp, dtype=torch.float64).pin_memory()
    d = info["d1"] + info["d2"]
    hfine = torch.empty((prob.N, (prob.n_f + 1) ** 2), dtype=torch.float64).pin_memory()
    hcoarse = torch.empty((prob.N + 1, d), dtype=torch.float64).pin_memory()
    import ctypes as C
    L = _lib.lib()
    e2e_t = []
    for it in range(args.warmup + args.steps):
        stv = _lib.Stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = L.pint_parareal_solve(p.h, hu0.data_ptr(), hf.data_ptr(), ha.data_ptr(), eps, prob.N, 1e-3 * eps,
                                  200, hfine.data_ptr(), hcoarse.data_ptr(), C.byref(stv))
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
        _lib.check(s)           # NOT_CONVERGED is an error here too
    e2e_value = world * dofsteps / max_over_ranks(sum(e2e_t) / len(e2e_t), world)
    h2d = (hu0.numel() + hf.numel() + ha.numel()) * 8
    d2h = (hfine.numel() + hcoarse.numel()) * 8
    st = stats[-1]
    # roofline of the dominant kernel (the WR contractions)
    peaks, src = load_peaks()
    hot_ms = st.get("hot_ms", 0.0)
    hot_flops = st.get("hot_flops", 0.0)
    hot_launches = st.get("hot_launches", 0)
    achieved = (hot_flops / (hot_ms / 1e3) / 1e12) if hot_ms > 0 else None
    if args.precision == "fp64":
        roof = {"bound": "alu", "kernel": "k_wr_gemm (FP64 WR contractions)", "achieved": achieved,
                "peak": FP64_MEASURED_TFLOPS, "unit": "TFLOP/s",
                "frac": (achieved / FP64_MEASURED_TFLOPS) if achieved else None, "traffic": None,
                "peak_source": "measured cuBLAS DGEMM on GB300 (FP64 pipe)"}
    elif args.precision == "mixed":
        # TF32 dense peak = measured sustained BF16 x nominal TF32/BF16 ratio (1.1 / 2.25)
        pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")) * (1.1 / 2.25)
        tr = umma_traffic() if args.config == "c2" else None
        roof = {"bound": "tensor", "kernel": "k_wr_umma (tcgen05 kind::tf32 WR contractions)",
                "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": (achieved / pk) if achieved else None, "traffic": tr,
                "traffic_unit": "bytes per launch (ncu dram read+write, profiles/k_wr_umma_c2_mixed.md)",
                "peak_source": f"{src} bf16 sustained x 1.1/2.25 (TF32)",
                "mma_frac": (3 * achieved / pk) if achieved else None,
                "note": "achieved counts the algorithmic 2 M N K once; the hi/lo split issues 3 MMAs per "
                        "K step, so the tensor pipe runs mma_frac of its peak"}
    else:
        pk = 69.7
        roof = {"bound": "alu", "kernel": "k_wr_gemm32 (FP32 CUDA-core WR contractions)", "achieved": achieved,
                "peak": pk, "unit": "TFLOP/s", "frac": (achieved / pk) if achieved else None, "traffic": None,
                "peak_source": "measured torch FP32 SGEMM on GB300"}
    roof.update({"launches": hot_launches, "avg_launch_ms": (hot_ms / hot_launches) if hot_launches else None})
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": mixed_dtype(args),
        "data": "synthetic (seeded splitmix64 high-contrast channels/inclusions; paper fields unavailable)",
        "config": {"workload": workload_desc(prob), "T": p.T,
                   "d1": info["d1"], "d2": info["d2"], "gamma": info["gamma"],
                   "reduced_dof_steps_per_s": world * (info["d1"] + info["d2"]) * prob.N * prob.P / t_step,
                   "lambda_max22": info["lambda_max22"], "precision": args.precision,
                   "coarse_sweeps": ("FP64 in both solves" if args.coarse_fp64 or args.precision == "fp64" else
                                     "FP32 cluster in the low-precision solve, FP64 in the correction solve"),
                   "jump_norm": "FP64",
                   "refinement_residual": "FP64" if args.refine_fp64 else "double-float (~48 bits, FP32 pipe)",
                   "status": st["status"], "converged": all(s["converged"] for s in stats),
                   "K1": st["K1"], "wr_total": st["wr_total"], "wr_iters": st["wr_iters"],
                   "rel_l2_vs_fp64_max_t": rel_err, "fp64_gpu_value": dofsteps / (st64["solve_ms"] / 1e3),
                   "fp64_gpu_ms": st64["solve_ms"], "fp64_K1": st64["K1"], "fp64_wr_total": st64["wr_total"],
                   "setup_s": setup_s,
                   "setup_stages_s": dict(zip(("block_eigenproblems", "oversampled_bases", "galerkin", "reduced",
                                               "spectral", "time_grid"), stages)),
                   "l2": "512 MB buffer zeroed before every timed step",
                   "contraction_tiles": ("cost model" if args.no_autotune or args.precision != "mixed" else
                                         [{k: r[k] for k in ("M", "ncols", "tn", "s", "pair", "us")}
                                          for r in api.tuning_table()]),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clk.summary(),
        "split_ms": {"f": st["f_ms"], "g": st["g_ms"], "prolong": st["prolong_ms"]},
    }
    p.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.config, prob)
    return out


def run_reference(args, rank, world):
    """The oracle timed on the host cores, each step a bounded sample of the
    workload (the 64x64 workload: a complete solve per step)."""
    if rank != 0:
        return None
    if args.config not in ("c1", "c2"):
        return {"impl": "reference", "unavailable": "the oracle's timed sample is defined for the 64x64 and "
                                                    "256x256 workloads only"}
    prob = problem(args.config)
    smp = OracleSampler(args.config, prob)
    dofsteps = smp.D * prob.N * prob.P
    secs, desc = [], ""
    # each step a bounded sample, sized so the whole run ends within a few minutes
    budget = max(1.0, 120.0 / max(1, args.warmup + args.steps))
    nsub = 1
    if args.config == "c2":
        t1, _, _ = smp.units(1)
        nsub = int(max(1, min(prob.N, budget / max(t1, 1e-3) / 2)))
    for it in range(args.warmup + args.steps):
        if args.config == "c1":
            t, st = smp.full_solve()
            desc = (f"one complete oracle solve per step (K1={st['K1']}, sum K0={sum(st['wr_iters'])}), "
                    f"{smp.cores} threads, setup excluded ({smp.setup_s:.1f} s)")
        else:
            t, desc = smp.sample(nsub)
        if it >= args.warmup:
            secs.append(t)
    t = statistics.mean(secs)
    v = dofsteps / t
    cb = {"value": v, "unit": UNIT, "cores": smp.cores, "kind": "oracle", "sample": desc}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(prob)},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def run_adjoint(args, rank, world):
    """The 128x128 adjoint workload: one step = pint_adjoint (the forward solve,
    the observation residuals, the backward parareal sweep and the gradients
    with respect to u0 and the 32 per-interval amplitudes).  value = fine
    unknowns x N P / time of the gradient call."""
    import torch
    from paper_2411_09244_gb300 import api, _lib, inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    prob = inputs.config_c3()
    obs = inputs.observation_nodes(prob.n_f, 64, seed=prob.n_f)
    data = np.random.default_rng(21).standard_normal((prob.N, obs.size))
    prec = {"fp64": _lib.PINT_FP64, "mixed": _lib.PINT_MIXED, "mixed_f32": _lib.PINT_MIXED_F32}[args.precision]
    t0 = time.perf_counter()
    p = api.from_problem(prob, device=dev, precision=prec)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    u0 = torch.tensor(prob.u0, dtype=torch.float64, device=dev)
    f = torch.tensor(prob.f, dtype=torch.float64, device=dev)
    amp = torch.tensor(prob.amp, dtype=torch.float64, device=dev)
    dd = torch.tensor(data, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        p.adjoint(obs, dd, u0, f, amp, eps=prob.eps)
    torch.cuda.synchronize()
    times = []
    barrier(world)
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            J, gu, ga = p.adjoint(obs, dd, u0, f, amp, eps=prob.eps)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    t = max_over_ranks(sum(times) / len(times), world)
    work = (prob.n_f - 1) ** 2 * prob.N * prob.P
    p.close()
    if rank != 0:
        return None
    return {"metric": METRIC + " (adjoint: gradient of the observation misfit)", "value": world * work / t,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "tf32x3/f32 forward, f32 transposed sweeps",
                      "mixed_f32": "f32"}[args.precision],
            "data": "synthetic (seeded splitmix64 channels, Gaussian bumps, 64 seeded observation nodes)",
            "config": {"workload": workload_desc(prob) + ", 64 observation nodes, gradient w.r.t. u0 and 32 "
                                                       "per-interval amplitudes", "T": p.T, "misfit": J,
                       "setup_s": setup_s, "l2": "512 MB buffer zeroed before every timed step",
                       "amplitude_gradient": "fine adjoint recomputed inside each interval"},
            "clocks": clk.summary()}


def run_batch(args, rank, world):
    """Many independent uneven instances (the many-instance recipe) solved at
    once by pint_batch_solve: one context and CUDA stream per instance, the
    library's worker threads.  value = sum over instances of D N P / device
    time of the batch; one-at-a-time solves of the same instances are
    reported beside it."""
    import torch
    from paper_2411_09244_gb300 import api, _lib, inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    sizes = tuple(int(x) for x in args.batch_sizes.split(","))
    # instances of this rank (weak scaling: each rank its own seeded block)
    probs = [inputs.config_c4(i, sizes=sizes) for i in batch_instances(rank, args.batch)]
    prec = {"fp64": _lib.PINT_FP64, "mixed": _lib.PINT_MIXED, "mixed_f32": _lib.PINT_MIXED_F32}[args.precision]
    t0 = time.perf_counter()
    pints, refs = [], []
    for prob in probs:
        s = torch.cuda.Stream(dev)
        with torch.cuda.stream(s):
            p = api.Pint(prob.n_f, prob.kappa, device=dev)
            p.build_multiscale_spaces(prob.nc, prob.J, prob.ell)
            p.assemble_reduced(None, prob.N, prob.P, prob.alpha, _lib.PINT_FP64)
            _, fine64, _ = p.parareal_solve(prob.u0, prob.f, prob.amp, eps=prob.eps)
            refs.append(fine64)
            if prec != _lib.PINT_FP64:
                p.assemble_reduced(p.T, prob.N, prob.P, prob.alpha, prec, autotune=not args.no_autotune)
        pints.append(p)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    work = sum((pr.n_f - 1) ** 2 * pr.N * pr.P for pr in probs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cur = torch.cuda.current_stream(dev)

    def timed(fn):
        # device time from an event before the first instance's launches to the
        # end of the last instance's stream (instance streams wait on e0)
        flush.zero_()                           # L2 flush between timed iterations
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for p in pints:
            p.stream.wait_event(e0)
        r = fn()
        for p in pints:
            cur.wait_stream(p.stream)
        e1.record(cur)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    def sequential():
        out = []
        for p, prob in zip(pints, probs):
            with torch.cuda.stream(p.stream):
                out.append(p.parareal_solve(prob.u0, prob.f, prob.amp, eps=prob.eps, want_fine=True))
        return out

    plan = api.BatchPlan(pints, probs, want_fine=True)

    def concurrent():
        return plan.run(args.workers)

    for _ in range(args.warmup):
        timed(sequential)                       # first: the autotuner times each shape alone
        timed(concurrent)
    torch.cuda.synchronize()
    tc, ts, launches = [], [], 0
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            t, res = timed(concurrent)
            tc.append(t)
            launches += sum(r[2]["launches"] for r in res)
        for _ in range(args.steps):
            ts.append(timed(sequential)[0])
    barrier(world)
    t_conc = max_over_ranks(sum(tc) / len(tc), world)
    t_seq = max_over_ranks(sum(ts) / len(ts), world)
    # end to end through pint_batch_solve with pinned host buffers (copies inside)
    hplan = api.BatchPlan(pints, probs, want_fine=True, host=True)
    e2e_t = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hplan.run(args.workers)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_value = world * work / max_over_ranks(sum(e2e_t) / len(e2e_t), world)
    rel, rel_t = 0.0, 0.0
    for (c, fine, st), ref in zip(res, refs):
        rel = max(rel, float(torch.linalg.norm(fine - ref) / torch.linalg.norm(ref)))
        for n in range(ref.shape[0]):
            nr = float(torch.linalg.norm(ref[n]))
            if nr > 0:
                rel_t = max(rel_t, float(torch.linalg.norm(fine[n] - ref[n])) / nr)
    for p in pints:
        p.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": world * work / t_conc, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_conc * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": mixed_dtype(args),
            "data": "synthetic (seeded splitmix64 high-contrast fields, many-instance recipe)",
            "config": {"workload": f"many-instance batch: {args.batch} instances per GPU, fine grids from {sizes}, "
                                   f"8-cell blocks, J 2-4, contrast 10^U(3,6), N in (16,32,64), P=32, ell=2",
                       "instances": [{"n_f": pr.n_f, "J": pr.J, "N": pr.N, "K1": r[2]["K1"],
                                      "wr_total": r[2]["wr_total"]} for pr, r in zip(probs, res)],
                       "sequential_ms": t_seq * 1e3, "sequential_value": world * work / t_seq,
                       "l2": "512 MB buffer zeroed before every timed step",
                       "rel_l2_vs_fp64": rel, "rel_l2_vs_fp64_max_t": rel_t, "setup_s": setup_s,
                       "accuracy_note": "rel_l2_vs_fp64: over each instance's whole trajectory, max over "
                                        "instances; _max_t: per coarse time (u0 = 0, so the first states "
                                        "are orders of magnitude below the solver's state scale)",
                       "schedule": f"pint_batch_solve: one context and CUDA stream per instance, "
                                   f"{args.workers or min(args.batch, 16)} library worker threads taking the longest "
                                   "instance first; contraction tiles per shape "
                                   + ("from the launch cost model" if args.no_autotune else
                                      f"measured by the autotuner ({len(api.tuning_table())} shapes)"),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": hplan.h2d_bytes,
                    "d2h_bytes_per_step": hplan.d2h_bytes},
            "clocks": clk.summary(), "gpu_launches": launches}


def main():
    args = parse()
    rank, world = dist_init(args)
    if args.tuning and args.impl != "reference" and os.path.exists(args.tuning):
        from paper_2411_09244_gb300 import api
        api.load_tuning(args.tuning)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.config == "c4":
        out = run_batch(args, rank, world)
    elif args.config == "c3":
        out = run_adjoint(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if args.tuning and args.impl != "reference" and rank == 0:
        from paper_2411_09244_gb300 import api
        api.save_tuning(args.tuning)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
