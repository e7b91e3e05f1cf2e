#!/usr/bin/env python
"""Benchmark of the MHAR walker step on one GB300 (or N replicas, one per GPU).

One bench step = one full run of the workload: z = 4096 walkers advanced
2000 iterations of Algorithm 2 on a random polytope with n = 100, m = 2000
(unit-norm Gaussian rows, b = 1, x0 = 0), in the mixed tensor-core mode, with
the final points written to a device buffer.  Metric: walker-steps/s
(= z x iterations / time, the paper's "samples per second" of Section 6.2).

The same line carries the mixing side of the metric ("ess"): on the
ill-conditioned random polytope (n = 500, m = 10000, axes scaled by s with
log s ~ U[ln 1e-3, 0], z = 16384) it times a learned-preconditioner run (500
warm-up iterations in four fit rounds, rank-32 + diagonal fit on the device,
then 5000 frozen iterations, tensor-core recompute mode) against plain isotropic runs (FP32 on
CUDA cores, and the same tensor-core mode), each with 500 + 5000 iterations,
and reports min-ESS (over coordinates, from a trace of 64 walkers every 5th
iteration, scaled to all z walkers) per second of device time -- for arms
whose split R_hat says they have left their transient; every arm also reports
R_hat and how far it has spread along each axis.  "ess_moderate" repeats it on
a smaller body (n = 40, m = 400, axes from 1e-2 to 1, z = 4096, 20000
iterations) whose long axes the warm-up reaches.

A third leg ("batched") times 256 random polytopes of different sizes (n
uniform in 20..400, m uniform in 2n..20n, z = 512 each, 1000 iterations)
advanced together by one kernel launch per iteration, with the cluster size
chosen by the library's autotuner.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2104_07097_gb300 import workloads as wl  # noqa: E402

WORKLOADS = {
    "rand100x2000": dict(name="rand100x2000", kind="random", n=100, m=2000, seed=2, z=4096,
                         iterations=2000),
    # The ill-conditioned body of the ESS leg, as a throughput workload.
    "illcond500x10000": dict(name="illcond500x10000", kind="illcond", n=500, m=10000, seed=5,
                             z=16384, iterations=200),
}
WORKLOAD = dict(WORKLOADS["rand100x2000"])
METRIC = "walker-steps/s"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu --set full capture of this workload (the
# commands are in profiles/); cold-cache per launch, as ncu replays it.  An
# entry must be dropped when its kernel changes.
PROFILED_TRAFFIC = {
    ("rand100x2000", "recompute_ts_kernel"): 9.575e6 + 0.0,
    ("illcond500x10000", "recompute_sk_kernel"): 127.926e6 + 30.817e6,
}
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE = dict(walkers=256, iterations=200)
BATCH_WORKLOAD = dict(name="batch256", count=256, seed=4, z=512, iterations=1000, tune_iters=8)
ESS_WORKLOAD = dict(name="illcond500x10000", n=500, m=10000, seed=5, smin=1e-3, z=16384,
                    warmup=500, iterations=5000, trace_walkers=64, trace_every=5, rank=32,
                    fit_rounds=4, snapshots=5, power_iters=4)
# A smaller ill-conditioned body whose long axes the 500 warm-up iterations do
# reach, run long enough (20000 iterations) for a chain to leave its transient,
# so that an ESS can be taken and the learned directions' effect on it shows.
ESS_MODERATE = dict(name="illcond40x400", n=40, m=400, seed=5, smin=1e-2, z=4096, warmup=500,
                    iterations=20000, trace_walkers=64, trace_every=5, rank=32, fit_rounds=4,
                    snapshots=5, power_iters=4)
REF_SAMPLE = dict(walkers=64, iterations=20)
RHAT_LIMIT = 1.05


def polytope():
    if WORKLOAD["kind"] == "illcond":
        return wl.ill_conditioned(WORKLOAD["n"], WORKLOAD["m"], seed=WORKLOAD["seed"])
    return wl.random_polytope(WORKLOAD["n"], WORKLOAD["m"], seed=WORKLOAD["seed"])


def config(precision: str) -> dict:
    return {"workload": f"{WORKLOAD['name']} z={WORKLOAD['z']} x {WORKLOAD['iterations']} iterations",
            "n": WORKLOAD["n"], "m": WORKLOAD["m"], "z": WORKLOAD["z"],
            "iterations_per_step": WORKLOAD["iterations"], "precision": precision,
            "l2": "flushed between steps (256 MiB write); the chain's own state stays resident within a step"}


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "_source": "fallback"}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mhar_bench_clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


def _oracle_shard(args):
    """One process of the all-cores oracle run: walkers w0 .. w0 + count - 1."""
    A, b, x0, count, w0, steps = args
    import oracle
    t0 = time.perf_counter()
    oracle.mhar_run(A, b, np.tile(x0, (count, 1)), steps=steps, thin=0, seed=0, walker0=w0)
    return time.perf_counter() - t0


def cpu_baseline(p) -> dict:
    """The FP64 oracle as it stands on the host's cores: one process per core
    (started with spawn), each on its own range of walkers (walkers are
    independent and the generator is counter-based, so the shards are one
    ensemble), and the same single-threaded run on one core."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    zs, ts = CPU_SAMPLE["walkers"], CPU_SAMPLE["iterations"]
    t0 = time.perf_counter()
    oracle.mhar_run(p.A, p.b, np.tile(p.x0, (zs, 1)), steps=ts, thin=0, seed=0)
    dt1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    jobs = [(p.A, p.b, p.x0, zs, k * zs, ts) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_shard, jobs[:1])          # start-up (imports, library load)
        t0 = time.perf_counter()
        pool.map(_oracle_shard, jobs)
        dtn = time.perf_counter() - t0
    return {"value": cores * zs * ts / dtn, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {zs} walkers x {ts} iterations of {WORKLOAD['name']} "
                      f"(FP64 oracle, disjoint walker ranges, {dtn:.1f} s wall)",
            "single_core": {"value": zs * ts / dt1, "cores": 1,
                            "sample": f"{zs} walkers x {ts} iterations, 1 thread, {dt1:.1f} s"}}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    p = polytope()
    zs, ts = REF_SAMPLE["walkers"], REF_SAMPLE["iterations"]
    X = np.tile(p.x0, (zs, 1))
    step0 = 0
    for _ in range(args.warmup):
        X = oracle.mhar_run(p.A, p.b, X, steps=ts, thin=0, seed=0, step0=step0)["X"]
        step0 += ts
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        X = oracle.mhar_run(p.A, p.b, X, steps=ts, thin=0, seed=0, step0=step0)["X"]
        times.append(time.perf_counter() - t0)
        step0 += ts
    ms = 1e3 * statistics.mean(times)
    value = zs * ts / (ms / 1e3)
    sample = f"{zs} walkers x {ts} iterations of {WORKLOAD['name']} per step (FP64 oracle, 1 thread)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random polytope)", "config": config("fp64-oracle"),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_leg(stream, torch, mhar, peaks) -> dict:
    """256 random polytopes (n ~ U{20..400}, m ~ U{2n..20n}), z = 512 each, one
    kernel launch per iteration for all of them (or one per bucket of similar
    n), launch shapes autotuned."""
    B = BATCH_WORKLOAD
    bodies = wl.batch(B["count"], seed=B["seed"])
    z, iters = B["z"], B["iterations"]
    t0 = time.perf_counter()
    bt = mhar.Batch([(p.A, p.b, p.x0) for p in bodies], z, seed=0, stream=stream)
    create_s = time.perf_counter() - t0
    try:
        C = bt.tune(B["tune_iters"])
        per_bucket, bucket_shapes, _ = bt.get_shapes()
        bt.run(16)  # warm-up with the chosen shape (graph capture)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        bt.run(iters)
        b.record(stream)
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        worst = max(bt.check(q).max_violation for q in range(len(bodies)))
        # Untimed: an FP64 audit of every problem's first 256 walkers after
        # each of 200 more iterations.
        bt.set_audit(1, 256)
        bt.run(200)
        audited = max(bt.check(q).run_max_violation for q in range(len(bodies)))
    finally:
        bt.close()
    flops = 4.0 * sum(p.m * p.n for p in bodies) * z * iters
    peak = peaks["bf16_tflops_sustained"]
    return {"workload": f"{B['name']}: {B['count']} random polytopes, n ~ U{{20..400}}, "
                        f"m ~ U{{2n..20n}}, z={z} each, {iters} iterations",
            "value": B["count"] * z * iters / secs, "unit": METRIC,
            "seconds": secs,
            "shape": ({"per_bucket": [c for c in bucket_shapes]} if per_bucket else C),
            # a chord kernel and a walker update per bucket (per batch)
            "launches_per_iteration": 2 * (sum(1 for c in bucket_shapes if c >= 0) if per_bucket else 1),
            "create_seconds": create_s,
            "roofline": {"bound": "tensor", "achieved": flops / secs / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": flops / secs / 1e12 / peak,
                         "frac_pipe": 3 * flops / secs / 1e12 / peak,
                         "algorithmic": "4 m n flops per walker-step (A x and A d); frac_pipe "
                                        "counts the 12 m n of the FP16x3 products"},
            "max_violation": worst,
            "audit": {"iterations": 200, "walkers_per_problem": 256,
                      "run_max_violation": audited}}


def configs_leg(stream, torch, mhar, peaks) -> dict:
    """Throughput on the remaining configurations: the hypercube in FP64 and the
    simplex with cuts (one equality) in the recompute tensor-core mode."""
    legs = {}
    cases = (
        ("cube10_fp64", wl.cube(10), 100, 1000, "fp64"),
        ("simplex1000+4000cuts_mixed_rs", wl.simplex_cuts(1000, 4000, seed=3), 8192, 1000,
         "mixed_rs"),
    )
    for name, p, z, iters, prec in cases:
        with mhar.Sampler(p.A, p.b, p.x0, z, AE=p.AE, bE=p.bE, precision=prec, seed=0,
                          stream=stream) as smp:
            smp.run(20)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            smp.run(iters)
            b.record(stream)
            torch.cuda.synchronize()
            secs = a.elapsed_time(b) / 1e3
            st = smp.check()
            leg = {"workload": f"{name}: n={p.n}, m={p.m}, m_E={p.mE}, z={z}, {iters} iterations",
                   "value": z * iters / secs, "unit": METRIC, "seconds": secs,
                   "kernel": smp.kernel_name(), "max_violation": st.max_violation,
                   "eq_residual": st.eq_residual}
            if prec == "mixed_rs":
                flops = 4.0 * p.m * p.n * z * iters
                pk = peaks["bf16_tflops_sustained"]
                leg["roofline"] = {"bound": "tensor", "achieved": flops / secs / 1e12,
                                   "peak": pk, "unit": "TFLOP/s", "frac": flops / secs / 1e12 / pk,
                                   "frac_pipe": 3 * flops / secs / 1e12 / pk,
                                   "note": "whole iteration incl. direction draw and projection; "
                                           "4 m n flops per walker-step (frac_pipe: 12 m n)"}
            smp.set_audit(1, min(z, 1024))
            smp.run(100)
            sa = smp.stats()
            leg["audit"] = {"iterations": 100, "walkers": min(z, 1024),
                            "run_max_violation": sa.run_max_violation,
                            "run_eq_residual": sa.run_eq_residual}
            legs[name] = leg
    return legs


def ess_leg(stream, torch, mhar, peaks, E=ESS_WORKLOAD) -> dict:
    """min-ESS/s of learned-preconditioned vs plain MHAR on an ill-conditioned body."""
    from paper_2104_07097_gb300 import diagnostics
    p = wl.ill_conditioned(E["n"], E["m"], seed=E["seed"], smin=E["smin"])
    z, T, W, every = E["z"], E["iterations"], E["trace_walkers"], E["trace_every"]
    out = torch.empty((T // every, W, p.n), dtype=torch.float64, device="cuda")
    arms = {}
    kernel_roofline = None
    # The first warm-up round of the learned arm walks with directions scaled
    # by the coordinates' extents read off the constraints, 1 / max_i |a_ij|
    # (a fixed diagonal law); every fit round then refits rank-32 + diagonal
    # from the chain's own warm-up points.
    extent = 1.0 / np.abs(p.A).max(axis=0)
    diag0 = extent / extent.max()
    for name, prec, learned in (("learned_mixed_rs", "mixed_rs", True),
                                ("plain_mixed_rs", "mixed_rs", False),
                                ("plain_fp32", "fp32", False)):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision=prec, seed=0, stream=stream,
                          out_on_device=True, emit_walkers=W) as smp:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            if learned:
                smp.set_preconditioner(diag0)
                # Each round warms up with the previous round's directions and refits.
                for _ in range(E["fit_rounds"]):
                    smp.fit_preconditioner(E["warmup"] // E["fit_rounds"], E["snapshots"],
                                           E["rank"], E["power_iters"])
            else:
                smp.run(E["warmup"])
            smp.run(T, thin=every, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            secs = a.elapsed_time(b) / 1e3
            st = smp.check()
            if name == "plain_mixed_rs":
                kms = smp.time_kernels(16)
                flops = 4.0 * p.m * p.n * z
                pk = peaks["bf16_tflops_sustained"]
                kernel_roofline = {
                    "bound": "tensor", "kernel": smp.kernel_name(),
                    "ms_per_iteration": kms[1],
                    "achieved": flops / (kms[1] * 1e-3) / 1e12,
                    "peak": pk, "unit": "TFLOP/s",
                    "frac": flops / (kms[1] * 1e-3) / 1e12 / pk,
                    "frac_pipe": 3 * flops / (kms[1] * 1e-3) / 1e12 / pk,
                    "algorithmic": "4 m n flops per walker-step (A x, A d); frac_pipe counts "
                                   "the 12 m n of the FP16x3 products"}
            # Untimed: FP64 audit of 1024 walkers after each of 200 more iterations.
            smp.set_audit(1, min(z, 1024))
            smp.run(200)
            audited = smp.stats().run_max_violation
        trace = out.cpu().numpy()
        ess = diagnostics.ess_per_coordinate(trace) * (z / W)
        rhat = diagnostics.split_rhat(trace)
        converged = bool(rhat.max() < RHAT_LIMIT)
        # How far the chains have spread along every axis: the walkers' spread
        # of x_j over the last quarter of the trace, in units of the axis
        # extent 1 / max_i |a_ij| read off the constraints.
        spread = trace[-max(1, trace.shape[0] // 4):].reshape(-1, p.n).std(axis=0) / extent
        arms[name] = {"min_ess": float(ess.min()) if converged else None,
                      "median_ess": float(np.median(ess)) if converged else None,
                      "min_ess_transient": float(ess.min()),
                      "seconds": secs,
                      "min_ess_per_s": float(ess.min()) / secs if converged else None,
                      "walker_steps_per_s": z * (E["warmup"] + T) / secs,
                      "max_split_rhat": float(rhat.max()),
                      "converged": converged,
                      "min_axis_spread": float(spread.min()),
                      "median_axis_spread": float(np.median(spread)),
                      "max_violation": st.max_violation,
                      "audit": {"iterations": 200, "walkers": min(z, 1024),
                                "run_max_violation": audited}}
    return {"workload": f"{E['name']} (axes scaled by s, log s ~ U[ln {E['smin']:g}, 0]) z={z}: "
                        f"{E['warmup']} warm-up + {T} iterations",
            "trace": f"{W} walkers, every {every}th iteration; ESS scaled by z/{W}; Geyer initial "
                     f"monotone sequence",
            "learned": f"rank {E['rank']} + diagonal, fitted on the device in {E['fit_rounds']} rounds "
                       f"of {E['warmup'] // E['fit_rounds']} warm-up iterations ({E['snapshots']} "
                       f"snapshots, {E['power_iters']} power iterations each), then frozen; the "
                       f"first round's directions are scaled by 1 / max_i |a_ij|; warm-up and "
                       f"fits are inside the timed region",
            "convergence": f"split R_hat over coordinates < {RHAT_LIMIT} (trace of the "
                           f"{T} iterations after warm-up); an arm that has not converged is "
                           f"still in its transient and reports no ESS (min_ess_transient is "
                           f"the estimator's value on it, not an ESS)",
            "axis_spread": "std over walkers and the last quarter of the trace of x_j, divided "
                           "by the axis extent 1 / max_i |a_ij|; min and median over j",
            "arms": arms,
            "roofline": kernel_roofline,
            "min_ess_per_s_learned_vs_plain_fp32": _ratio(arms, "min_ess_per_s"),
            "min_axis_spread_learned_vs_plain_fp32": _ratio(arms, "min_axis_spread")}


def _ratio(arms, key):
    a, b = arms["learned_mixed_rs"][key], arms["plain_fp32"][key]
    return a / b if a is not None and b else None


FEAS_TOL = 1e-6   # max(A x - b) <= FEAS_TOL |b|_inf; |b|_inf = 1 on every workload here


def mark_feasibility(node) -> bool:
    """Flags every leg (a dict carrying max_violation or run_max_violation)
    with "feasible": its measured and audited violations within FEAS_TOL;
    returns whether all legs are."""
    ok = True
    if isinstance(node, dict):
        for v in node.values():
            ok = mark_feasibility(v) and ok
        worst = [node[k] for k in ("max_violation", "run_max_violation")
                 if isinstance(node.get(k), (int, float))]
        audit = node.get("audit")
        if isinstance(audit, dict) and isinstance(audit.get("run_max_violation"), (int, float)):
            worst.append(audit["run_max_violation"])
        if worst and "max_violation" in node:
            node["feasible"] = bool(max(worst) <= FEAS_TOL)
            ok = ok and node["feasible"]
    return ok


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_rs", choices=["mixed_rs", "mixed", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ess", action="store_true", help="skip the min-ESS/s comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-polytope leg")
    ap.add_argument("--workload", default="rand100x2000", choices=sorted(WORKLOADS),
                    help="the timed workload (default: the headline random polytope)")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2104_07097_gb300 import build as libbuild
    from paper_2104_07097_gb300 import mhar
    # One rank per node compiles (if the library is stale); the others wait,
    # so no two processes write the same object files.
    if local == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()
    libbuild.build()
    mhar.load()

    p = polytope()
    z, iters = WORKLOAD["z"], WORKLOAD["iterations"]
    stream = torch.cuda.current_stream()
    s = mhar.Sampler(p.A, p.b, p.x0, z, precision=args.precision, seed=0, walker0=rank * z,
                     stream=stream, out_on_device=True)
    out = torch.empty((1, z, p.n), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(3, args.warmup)):
        s.run(iters, thin=iters, out=out)
    torch.cuda.synchronize()
    launches0 = s.stats().kernel_launches

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            s.run(iters, thin=iters, out=out)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    launches = s.stats().kernel_launches - launches0
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * z * iters / (ms / 1e3)

    # Per-kernel device times (CUDA events around each launch, same stream).
    kms = s.time_kernels(128)
    st = s.check()
    # Untimed: an FP64 audit of 1024 walkers after each of 256 more iterations.
    s.set_audit(1, min(z, 1024))
    s.run(256)
    audited = s.stats().run_max_violation
    s.set_audit(0, 0)
    peaks = load_peaks()
    m, n = p.m, p.n
    if args.precision in ("mixed", "mixed_rs"):
        # The method's own work per walker-step: A d (2 m n flops) in the
        # stored-slack mode, A x and A d (4 m n) in the recompute mode.  The
        # tensor pipe runs FP16 products of 2 m n each: 4 (stored) or 6
        # (recompute), reported as frac_pipe.
        nmeth, nprod = (1, 4) if args.precision == "mixed" else (2, 6)
        flops = 2.0 * nmeth * m * n * z
        pipe = 2.0 * nprod * m * n * z
        peak = peaks["bf16_tflops_sustained"]
        sec = kms[1] * 1e-3
        roofline = {"bound": "tensor", "achieved": flops / sec / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / sec / 1e12 / peak,
                    "frac_pipe": pipe / sec / 1e12 / peak,
                    "traffic": PROFILED_TRAFFIC.get((WORKLOAD["name"], s.kernel_name())),
                    "kernel": s.kernel_name(),
                    "algorithmic": f"{2 * nmeth} m n flops per walker-step (the method's "
                                   f"products); frac_pipe counts the {2 * nprod} m n flops of "
                                   f"its {nprod} FP16 products",
                    "peak_source": f"{peaks['_source']} bf16 sustained (FP16 rate = BF16 rate)"}
    else:
        bytes_ = 2.0 * m * n * z * (8 if args.precision == "fp64" else 4)
        roofline = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                    "traffic": None, "kernel": s.kernel_name()}

    # End to end through the public API from pinned host buffers: create
    # (H2D of A, b, x0), run, D2H of the emitted points, destroy.
    pinA = torch.from_numpy(p.A).pin_memory()
    pinb = torch.from_numpy(p.b).pin_memory()
    pinx = torch.from_numpy(p.x0).pin_memory()
    pinout = torch.empty((1, z, n), dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(min(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mhar.Sampler(pinA.numpy(), pinb.numpy(), pinx.numpy(), z, precision=args.precision,
                          seed=1, walker0=rank * z, stream=stream) as se:
            se.run(iters, thin=iters, out=pinout.numpy())
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * z * iters / e2e_s, "unit": METRIC,
           "h2d_bytes_per_step": int(8 * (m * n + m + n)), "d2h_bytes_per_step": int(8 * z * n + 16)}

    # Plain FP32 MHAR (CUDA cores, the paper's recompute formulation) on the
    # same workload, for the mixed-vs-plain comparison.
    plain = None
    if args.precision in ("mixed", "mixed_rs"):
        with mhar.Sampler(p.A, p.b, p.x0, z, precision="fp32", seed=0, walker0=rank * z,
                          stream=stream, out_on_device=True) as sp:
            sp.run(iters, thin=iters, out=out)
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            sp.run(iters, thin=iters, out=out)
            b2.record(stream)
            torch.cuda.synchronize()
            plain = {"value": z * iters / (a.elapsed_time(b2) / 1e3), "unit": METRIC,
                     "precision": "fp32 (CUDA cores)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "f16x4-f32acc", "mixed_rs": "f16x3-f32acc", "fp32": "f32",
                          "fp64": "f64"}[args.precision],
                "data": "synthetic (seeded random polytope, unit-norm Gaussian rows)",
                "config": config(args.precision), "roofline": roofline,
                "kernel_ms": {"directions": kms[0], "chord": kms[1], "refresh": kms[2]},
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
                "feasibility": {"max_violation": st.max_violation, "refresh_drift": st.refresh_drift,
                                "stalls": st.stalls,
                                "audit": {"iterations": 256, "walkers": min(z, 1024),
                                          "run_max_violation": audited}},
                "plain_fp32": plain}
        if world == 1 and not args.no_batch and args.precision == "mixed_rs":
            line["batched"] = batch_leg(stream, torch, mhar, peaks)
            line["other_configs"] = configs_leg(stream, torch, mhar, peaks)
        if world == 1 and not args.no_ess:
            line["ess"] = ess_leg(stream, torch, mhar, peaks)
            line["ess_moderate"] = ess_leg(stream, torch, mhar, peaks, ESS_MODERATE)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p)
        line["feasibility_ok"] = mark_feasibility(line)
        if not line["feasibility_ok"]:
            print("bench: a leg broke max(A x - b) <= 1e-6 |b|_inf (see its 'feasible' flag)",
                  file=sys.stderr)
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
