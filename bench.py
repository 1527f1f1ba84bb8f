#!/usr/bin/env python
"""Benchmark of the tiled-QR least-squares path on one GB300 (per rank).

Workload: min ||A x - b|| for A = U diag(sigma) V^T, 32768 x 4096, cond 1e6 (Haar U, V;
geometric sigma), x ~ N(0,1), b = A x + 1e-3 N(0,1), seeded; one right-hand side.

One step = one call of the library's least-squares entry point (tqr_lstsq):
  mixed (headline): FP32 copy of A -> elimination list + task graph (cached plan) ->
    tiled QR (GEQRT/TTQRT panels with FP64 norms and tau, UNMQR/TTMQR on tcgen05 with
    split-bf16 x3 products, one persistent kernel) -> FP64 refinement (residuals, A^T r,
    LSQR preconditioned by R) until the LS optimality ||A^T r|| / (||A||_F ||r||)
    reaches that of the plain FP64 solve ("equal LS error");
  fp64 arm: FP64 tiled QR (nb 256, ib 32) -> Q^T b -> triangular solve.
value = nominal 2 n^2 (m - n/3) flops per step / step time (TFLOP/s).  A is 1.07 GB,
larger than the 129 MB L2, so every step streams it from HBM.

--impl reference times the CPU oracle (plain numpy FP64, one thread) on a bounded sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tiled-QR TFLOP/s, mixed vs plain FP64 at equal LS error; % of tensor peak"
FP64_NOMINAL_TFLOPS = 1.25     # GB300's nominal FP64 rate (context; the fraction uses the measured one)
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz maximum SM clock
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
BATCH_COUNT = 2048
# DRAM bytes (read + write) per nominal flop of the two executors, from one ncu capture
# each of the unchanged kernels on smaller inputs of the same kind (the tensor-core
# executor, PlasmaTree-TS(16), on a 24576 x 2048 matrix: 7.527 GB for 2.004e11 nominal
# flops, traffic growing with the number of tile updates as the flops do; the batched FP32
# executor on the first 256 matrices of the batch: 1.317 GB for 4.907e10 flops).
MIXED_TRAFFIC_PER_FLOP = 7.527e9 / 2.004e11
BATCH_TRAFFIC_PER_FLOP = 1.317e9 / 4.907e10
BF16_FALLBACK = (1900.0, 1700.0)
# Kernel weights of the library's default claim order for the tensor-core precisions
# (tqr_set_claim_order mode 2 at nb 128, bf16x6: measured task durations with tuned panel
# weights), and the mean task durations (us) of the same executor from a per-task trace on
# GB300 (32768 x 4096, PlasmaTree-TS(16)), the weights of the schedule bound.  Order:
# GEQRT, TTQRT, UNMQR, TTMQR, TSQRT, TSMQR, operand-image preparation, TTQRT block, TSQRT
# block (the tensor-core graph splits its TT / TS panels into 32-column block tasks, so the
# whole-panel TTQRT / TSQRT weights do not occur in it).
TENSOR_CLAIM_WEIGHTS = (265, 285, 20, 32, 320, 32, 66, 80, 85)
TENSOR_TASK_MEAN_US = (205, 286, 22, 26, 270, 26, 62, 57, 67)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=32768)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--cond", type=float, default=1e6)
    ap.add_argument("--prec", default="bf16x6")
    ap.add_argument("--also-prec", default="bf16x3", help="second mixed precision measured for comparison ('' = none)")
    ap.add_argument("--no-trees", action="store_true",
                    help="skip the FP64 factorization under the six trees and their TS forms "
                         "(32768x4096, nb 256, ib 32; about 20 s)")
    ap.add_argument("--tree", default="plasma-ts", help="tree of the mixed arm (a '-ts' suffix: its TS form)")
    ap.add_argument("--bs", type=int, default=16, help="PlasmaTree domain size of the mixed arm")
    ap.add_argument("--fp64-tree", default="plasma-ts")
    ap.add_argument("--fp64-bs", type=int, default=16)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-m", type=int, default=8192)
    ap.add_argument("--sample-n", type=int, default=1024)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched measurement (2048 FP32 matrices, one launch)")
    ap.add_argument("--batch-prec", default="fp32")
    ap.add_argument("--batch-table", default="auto",
                    help="tuning table of the batch: 'auto' (the library's autotuner, tqr_batch_autotune), "
                         "'builtin' (the built-in size classes) or a JSON file with a 'table'")
    ap.add_argument("--batch-reps", type=int, default=5)
    ap.add_argument("--batch-tensor-prec", default="bf16x6",
                    help="also run the batch with this tensor-core precision ('' = no)")
    ap.add_argument("--no-c5", action="store_true",
                    help="skip the square 16384^2 solve (cond 1e4, 64 right-hand sides; about 1 min)")
    ap.add_argument("--c5-precs", default="bf16x3,bf16x6")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return BF16_FALLBACK[0], BF16_FALLBACK[1], "fallback"


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


# ---------------------------------------------------------------------------------
# CPU oracle timing (subprocess, one BLAS thread)
# ---------------------------------------------------------------------------------

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import synthetic
from oracle import elimlists as E, householder as H
m, n, nb, ib, tree, bs, reps = {m}, {n}, {nb}, {ib}, {tree!r}, {bs}, {reps}
A, X, B = synthetic.least_squares_problem(m, n, {cond}, 1e-3, 1, synthetic.SEED_BASE + 3)
p, q = H.tile_grid(m, n, nb)
TREES = dict(flat=E.FLAT, plasma=E.PLASMA, binary=E.BINARY, fibonacci=E.FIBONACCI, greedy=E.GREEDY,
             grasap=E.GRASAP, asap=E.ASAP)
ts = tree.endswith("-ts")
base = tree[:-3] if ts else tree
times = []
for r in range(reps):
    t0 = time.perf_counter()
    elims = E.elimination_list(p, q, TREES[base], bs=bs)
    H.lstsq(A, B, nb, ib, elims, ts)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(times=times, flops=2.0 * n * n * (m - n / 3.0))))
"""


def run_oracle(m, n, nb, ib, tree, bs, reps, cond, threads=1):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = ORACLE_SNIPPET.format(root=ROOT, m=m, n=n, nb=nb, ib=ib, tree=tree, bs=bs, reps=reps, cond=cond)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cpu():
    """(logical cores, CPU model name) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def cpu_baseline(args):
    """The oracle timed on a bounded sample of the workload: with every host core as BLAS
    threads (the value) and with one thread (beside it)."""
    ms, ns = min(args.sample_m, args.m), min(args.sample_n, args.n)
    cores, model = host_cpu()
    multi = run_oracle(ms, ns, 256, 32, args.fp64_tree, args.fp64_bs, 1, args.cond, threads=cores)
    one = run_oracle(ms, ns, 256, 32, args.fp64_tree, args.fp64_bs, 1, args.cond, threads=1)
    tm, t1 = multi["times"][0], one["times"][0]
    return {"value": multi["flops"] / tm / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"oracle FP64 tiled-QR least squares (nb 256, ib 32, {args.fp64_tree} bs {args.fp64_bs}) "
                      f"of a {ms}x{ns} matrix "
                      f"of the same kind, numpy with {cores} BLAS threads (nproc), {tm:.1f} s; rate = nominal "
                      f"flops / time",
            "single_thread": {"value": one["flops"] / t1 / 1e12, "unit": "TFLOP/s", "cores": 1, "seconds": t1}}


def workload_config(args):
    return {"workload": f"least squares {args.m}x{args.n}, cond {args.cond:g}, 1 rhs; mixed tiled QR "
                        f"({args.prec}, nb 128, ib 32, {args.tree} bs {args.bs}) + FP64 refinement vs FP64 "
                        f"tiled QR (nb 256, ib 32, {args.fp64_tree} bs {args.fp64_bs})",
            "m": args.m, "n": args.n, "cond": args.cond, "nrhs": 1, "prec": args.prec, "tree": args.tree,
            "bs": args.bs, "fp64_tree": args.fp64_tree, "fp64_bs": args.fp64_bs,
            "nb_mixed": 128, "nb_fp64": 256, "ib": 32,
            "l2": "inputs larger than L2 (A is %.2f GB FP64)" % (args.m * args.n * 8 / 1e9),
            "parallelism": "independent replicas" if args.gpus > 1 else "single GPU"}


def reference_arm(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    ms, ns = min(2048, args.m), min(512, args.n)
    r = run_oracle(ms, ns, 256, 32, args.fp64_tree, args.fp64_bs, args.warmup + args.steps, args.cond)
    times = r["times"][args.warmup:]
    tot = sum(times)
    value = r["flops"] * len(times) / tot / 1e12
    sample = (f"oracle FP64 tiled-QR least squares (nb 256, ib 32, {args.fp64_tree} bs {args.fp64_bs}) of a "
              f"{ms}x{ns} matrix of "
              f"the workload's kind per step, one BLAS thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------
# Batched factorization: 2048 FP32 matrices, rows U[256, 8192], columns {32..256}
# ---------------------------------------------------------------------------------

def batched_measurement(args, hbm_gbs, rank=0, world=1, device=None, prec=None):
    """One graph-replayed persistent launch over the whole batch vs the same plan
    without a graph vs one tqr_factor launch per matrix (device time, inputs restored
    untimed before each launch; the 4.2 GB batch is larger than L2).  With several
    ranks each takes every world-th matrix and the times are maxima over ranks."""
    import numpy as np
    import torch

    import paper_1303_3182_gb300 as tqr
    import synthetic
    from paper_1303_3182_gb300 import replicas
    from paper_1303_3182_gb300.autotune import DeviceBatch, size_classes, time_launch

    prec = prec or args.batch_prec
    all_shapes = synthetic.ragged_batch_shapes(BATCH_COUNT, seed=synthetic.SEED_BASE + 4)
    shapes = [all_shapes[b] for b in replicas.shard(len(all_shapes), rank, world)]
    ms, ns = [m for m, _ in shapes], [n for _, n in shapes]
    table, tuning, tune_s = None, "built-in size classes", 0.0
    if args.batch_table == "auto":
        import time
        t0 = time.perf_counter()
        table = tqr.batch_autotune([m for m, _ in all_shapes], [n for _, n in all_shapes], prec)
        tune_s = time.perf_counter() - t0
        tuning = "autotuned (tqr_batch_autotune: per size class, device-timed)"
    elif args.batch_table and args.batch_table != "builtin":
        with open(args.batch_table) as fh:
            table = json.load(fh)["table"]
        tuning = "table " + args.batch_table
    params = tqr.batch_params(ms, ns, prec, table)
    db = DeviceBatch(shapes, replicas.replica_seed(synthetic.SEED_BASE + 4, rank),
                     dtype=torch.float64 if prec == "fp64" else torch.float32)
    plan = tqr.BatchPlan(db.As, prec, params=params)
    info = plan.info()
    graph_ms = time_launch(plan, db.restore, reps=args.batch_reps, use_graph=True)
    plain_ms = time_launch(plan, db.restore, reps=max(2, args.batch_reps // 2), use_graph=False)
    # one launch per matrix (the same tuning, the same T buffers)
    off = tqr.batch_workspace_offsets(ms, ns, prec, params)
    Ts = [plan.T[int(off[b]):int(off[b + 1])] for b in range(len(shapes))]
    stream = torch.cuda.current_stream()

    def per_matrix():
        for b, A in enumerate(db.As):
            nb, ib, tree, bs = (int(x) for x in params[b])
            tqr.factor(A, nb, ib, tree, bs, prec, T=Ts[b], stream=stream)

    old = tqr.set_sync(False)
    db.restore()
    per_matrix()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    db.restore()
    e0.record(stream)
    per_matrix()
    e1.record(stream)
    torch.cuda.synchronize()
    tqr.set_sync(old)
    tqr.lib().tqr_sync_status(None)
    per_ms = e0.elapsed_time(e1)
    graph_ms, plain_ms, per_ms = replicas.max_over_ranks([graph_ms, plain_ms, per_ms], device)
    flops = sum(tqr.nominal_flops(m, n) for m, n in all_shapes)
    esz = 8 if prec == "fp64" else 4
    all_params = tqr.batch_params([m for m, _ in all_shapes], [n for _, n in all_shapes], prec, table)
    t_bytes = int(sum(tqr.workspace_size(m, n, int(p[0]), int(p[1]), prec) for (m, n), p in zip(all_shapes, all_params)))
    a_bytes = 2 * esz * sum(m * n for m, n in all_shapes)
    byts = a_bytes + t_bytes
    peak = FP32_ALU_PEAK_TFLOPS if prec == "fp32" else FP64_NOMINAL_TFLOPS
    classes = []
    all_ms = [m for m, _ in all_shapes]
    for (lo, hi, n), idx in sorted(size_classes(all_shapes).items()):
        f_c = sum(tqr.nominal_flops(all_ms[b], n) for b in idx)
        b_c = sum(2 * esz * all_ms[b] * n + tqr.workspace_size(all_ms[b], n, int(all_params[b][0]),
                                                               int(all_params[b][1]), prec) for b in idx)
        ai = f_c / b_c
        classes.append({"m": [lo, min(hi, max(all_ms))], "n": n, "matrices": len(idx), "flops": f_c,
                        "ai_flop_per_byte": ai, "bound_tflops": min(peak * world, ai * hbm_gbs * world / 1e3),
                        "nb": int(all_params[idx[0]][0]), "ib": int(all_params[idx[0]][1]),
                        "tree": int(all_params[idx[0]][2])})
    t_bound = max(flops / (peak * 1e12 * world), byts / (hbm_gbs * 1e9 * world)) * 1e3
    achieved = flops / (graph_ms * 1e-3) / 1e12
    plan.close()
    del db
    torch.cuda.empty_cache()
    return {
        "workload": f"batched QR of {BATCH_COUNT} {prec.upper()} matrices, rows uniform in [256, 8192], "
                    "columns uniform in {32, 64, 128, 256}, N(0,1), seed 1303318204",
        "metric": "nominal TFLOP/s of one batched launch", "value": achieved, "unit": "TFLOP/s",
        "ms_graph_launch": graph_ms, "ms_plain_launch": plain_ms, "ms_one_launch_per_matrix": per_ms,
        "speedup_vs_per_matrix": per_ms / graph_ms, "tasks": info["tasks"], "edges": info["edges"],
        "resident_ctas": info["slots"], "tuning": tuning, "tuning_seconds": tune_s,
        "table": [[int(x) for x in row] for row in table] if table is not None else None,
        "ranks": world, "scaling": "strong (the 2048 matrices split across ranks)",
        "roofline": {"bound": "alu" if flops / peak > byts / (hbm_gbs * 1e-3) else "hbm",
                     "peak_tflops": peak, "peak_source": "FP32 CUDA cores: 152 SMs x 128 lanes x 2 x 2.07 GHz"
                     if prec == "fp32" else "FP64 nominal", "hbm_gbs": hbm_gbs,
                     "algorithmic_bytes": byts, "flops": flops, "bound_ms": t_bound,
                     "traffic": flops * BATCH_TRAFFIC_PER_FLOP,
                     "traffic_note": "bytes per launch, ncu capture of 256 matrices scaled by nominal flops",
                     "frac": t_bound / graph_ms, "classes": classes},
        "l2": "inputs larger than L2 (%.2f GB), restored before every launch" % (a_bytes / 2 / 1e9),
    }


# ---------------------------------------------------------------------------------
# Small case: 512 x 128 FP64, nb 64, ib 16, Greedy - latency / critical-path bound
# ---------------------------------------------------------------------------------

def c1_measurement(reps=20):
    """Device time of one FP64 factorization of the 512 x 128 matrix (8 x 2 tiles of 64),
    against its weighted critical path (34 units of 64^3/3 flops: the work of 34 GEQRT-
    equivalents in a chain) - this size is bound by the task chain, not by a peak."""
    import torch

    import paper_1303_3182_gb300 as tqr
    import synthetic

    m, n, nb, ib = 512, 128, 64, 16
    A0 = torch.from_numpy(synthetic.gaussian(m, n, synthetic.SEED_BASE + 1).T.copy()).cuda().t()
    work = torch.empty_like(A0.t()).t()
    T = torch.empty(tqr.workspace_size(m, n, nb, ib, "fp64"), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    work.copy_(A0)
    tqr.factor(work, nb, ib, "greedy", 1, "fp64", T=T)
    ts = []
    for _ in range(reps):
        work.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tqr.factor(work, nb, ib, "greedy", 1, "fp64", T=T)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    cp = tqr.elimlist(m // nb, n // nb, "greedy", 1)[1]
    ms = ts[len(ts) // 2]
    return {"workload": "512x128 FP64 N(0,1), seed 1303318201, nb 64, ib 16, Greedy", "ms_median": ms,
            "cp_units": cp, "us_per_cp_unit": ms * 1e3 / cp, "tflops": tqr.nominal_flops(m, n) / (ms * 1e-3) / 1e12,
            "note": "includes the synchronizing status read of the call"}


# ---------------------------------------------------------------------------------
# Square solve: A = U diag(sigma) V^T 16384 x 16384, cond 1e4, 64 right-hand sides N(0,1)
# ---------------------------------------------------------------------------------

def c5_measurement(args, n=16384, nrhs=64, cond=1e4):
    """FP64 tiled QR solve (nb 256) vs tensor-core factorization (nb 128) + FP64
    refinement, both through tqr_lstsq; equal-error criterion for a square system: the
    normwise backward error ||b - A x|| / (||A||_F ||x|| + ||b||) of every right-hand
    side, worst case, must not exceed the FP64 solve's by more than 2x."""
    import torch

    import paper_1303_3182_gb300 as tqr
    import synthetic

    dev = torch.device("cuda")
    A = synthetic.conditioned_device(n, n, cond, synthetic.SEED_BASE + 5, dev)
    g = torch.Generator(device=dev)
    g.manual_seed(synthetic.SEED_BASE + 5 + 7919)
    B = tqr.colmajor(torch.randn(n, nrhs, dtype=torch.float64, device=dev, generator=g))
    anorm = float(torch.linalg.norm(A))
    bnorm = torch.linalg.norm(B, dim=0)
    flops = tqr.nominal_flops(n, n)
    stream = torch.cuda.current_stream()

    def backward_error(X):
        R = B - A @ X
        return float((torch.linalg.norm(R, dim=0) / (anorm * torch.linalg.norm(X, dim=0) + bnorm)).max())

    def timed(prec, nb, tol, reps):
        ws = torch.empty(tqr.lstsq_workspace_size(n, n, nrhs, nb, 32, prec), dtype=torch.uint8, device=dev)
        X = tqr.colmajor(torch.empty((n, nrhs), dtype=torch.float64, device=dev))
        it = tqr.lstsq(A, B, nb, 32, "greedy", 4, prec, tol=tol, max_iter=1000, X=X, workspace=ws, stream=stream,
                       return_iters=True)[1]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            tqr.lstsq(A, B, nb, 32, "greedy", 4, prec, tol=tol, max_iter=1000, X=X, workspace=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        err = backward_error(X)
        del ws
        torch.cuda.empty_cache()
        return {"prec": prec, "nb": nb, "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12, "backward_error": err,
                "refinement_iterations": it}

    out = {"workload": f"square solve {n}x{n}, cond {cond:g}, {nrhs} right-hand sides N(0,1), seed 1303318205; "
                       "Greedy, ib 32; FP64 nb 256 vs tensor-core nb 128 + FP64 refinement",
           "nominal_flops": flops}
    fp64 = timed("fp64", 256, 1e-14, 1)
    out["fp64"] = fp64
    out["mixed"] = []
    for prec in [p for p in args.c5_precs.split(",") if p]:
        # refined to the FP64 solve's backward error (the equal-error criterion), or until
        # an outer step no longer halves it
        r = timed(prec, 128, 2 * fp64["backward_error"], 2)
        r["speedup_vs_fp64"] = fp64["ms"] / r["ms"]
        r["equal_error"] = r["backward_error"] <= 2 * fp64["backward_error"]
        out["mixed"].append(r)
    return out


# ---------------------------------------------------------------------------------
# Double complex (the thesis's second precision): 8192 x 2048 N(0,1) complex matrix
# ---------------------------------------------------------------------------------

def z64_measurement(m=8192, n=2048, nb=128, ib=32, fp64_peak=None):
    """Device time of the double-complex tiled QR (TQR_Z64) under Greedy and the TS form of
    PlasmaTree(16); flops 4 x 2 n^2 (m - n/3) (a complex multiply-add is 8 real flops)."""
    import torch

    import paper_1303_3182_gb300 as tqr
    import synthetic

    g = torch.Generator(device="cuda")
    g.manual_seed(synthetic.SEED_BASE + 6)
    A0 = torch.randn(n, m, dtype=torch.complex128, device="cuda", generator=g).t()
    work = torch.empty_like(A0.t()).t()
    T = torch.empty(tqr.workspace_size(m, n, nb, ib, "z64"), dtype=torch.uint8, device="cuda")
    flops = 4.0 * tqr.nominal_flops(m, n)
    out = {"workload": f"double-complex tiled QR {m}x{n}, N(0,1) real and imaginary parts, seed 1303318206, "
                       f"nb {nb}, ib {ib}", "complex_flops": flops, "trees": {}}
    tqr.set_timing(True)
    for tree, bs in (("greedy", 1), ("plasma-ts", 16)):
        work.copy_(A0)
        tqr.factor(work, nb, ib, tree, bs, "z64", T=T)  # plan and warm-up
        work.copy_(A0)
        tqr.kernel_time("factor", reset=True)
        tqr.factor(work, nb, ib, tree, bs, "z64", T=T)
        ms = tqr.kernel_time("factor", reset=True)[0]
        r = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
        if fp64_peak:
            r["frac_of_fp64_peak"] = r["tflops"] / fp64_peak
        out["trees"][f"{tree}" + (f"({bs})" if tree.startswith("plasma") else "")] = r
    tqr.set_timing(False)
    del A0, work, T
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------

def main_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1303_3182_gb300 as tqr
    import synthetic
    from paper_1303_3182_gb300 import build as _build
    from paper_1303_3182_gb300 import replicas

    rank, local, world = replicas.env_ranks()
    torch.cuda.set_device(local)
    replicas.init("nccl", torch.device("cuda", local))
    _build.build()
    tqr.lib()
    dev = torch.device("cuda", local)
    m, n = args.m, args.n
    stream = torch.cuda.current_stream()
    # independent replicas: each rank solves its own seeded problem
    A, xtrue, b = synthetic.least_squares_device(m, n, args.cond, 1e-3, 1,
                                                 replicas.replica_seed(synthetic.SEED_BASE + 3, rank), dev)
    anorm = float(torch.linalg.norm(A))

    def optimality(X):
        r = b - A @ X
        return float(torch.linalg.norm(A.t() @ r) / (anorm * torch.linalg.norm(r)))

    X = tqr.colmajor(torch.empty((n, 1), dtype=torch.float64, device=dev))

    # ---- plain FP64 arm (the same entry point, FP64 tiled QR) ----
    ws64 = torch.empty(tqr.lstsq_workspace_size(m, n, 1, 256, 32, "fp64"), dtype=torch.uint8, device=dev)
    tqr.lstsq(A, b, 256, 32, args.fp64_tree, args.fp64_bs, "fp64", X=X, workspace=ws64, stream=stream)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.fp64_steps):
        tqr.lstsq(A, b, 256, 32, args.fp64_tree, args.fp64_bs, "fp64", X=X, workspace=ws64, stream=stream)
    g1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = g0.elapsed_time(g1) / args.fp64_steps
    eta64 = optimality(X)
    del ws64
    torch.cuda.empty_cache()

    # ---- mixed arm (headline) ----
    tol = eta64
    ws = torch.empty(tqr.lstsq_workspace_size(m, n, 1, 128, 32, args.prec), dtype=torch.uint8, device=dev)

    def step():
        return tqr.lstsq(A, b, 128, 32, args.tree, args.bs, args.prec, tol=tol, max_iter=1000, X=X, workspace=ws,
                         stream=stream, return_iters=True)[1]

    tqr.set_timing(True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for kind in ("factor", "apply_q", "trsm", "refine"):
        tqr.kernel_time(kind, reset=True)
    tqr.launch_count(reset=True)
    replicas.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            iters.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    replicas.barrier()
    ms_total = e0.elapsed_time(e1)
    launches = tqr.launch_count(reset=True)
    kt = {k: tqr.kernel_time(k, reset=True) for k in ("factor", "apply_q", "trsm", "refine")}
    tqr.set_timing(False)
    eta_mixed = optimality(X)

    # ---- second mixed precision (fewer steps, reported beside the headline) ----
    also = None
    if args.also_prec and args.also_prec != args.prec:
        ws2 = torch.empty(tqr.lstsq_workspace_size(m, n, 1, 128, 32, args.also_prec), dtype=torch.uint8,
                          device=dev)
        it2 = tqr.lstsq(A, b, 128, 32, args.tree, args.bs, args.also_prec, tol=tol, max_iter=1000, X=X, workspace=ws2,
                        stream=stream, return_iters=True)[1]
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(2):
            it2 = tqr.lstsq(A, b, 128, 32, args.tree, args.bs, args.also_prec, tol=tol, max_iter=1000, X=X,
                            workspace=ws2, stream=stream, return_iters=True)[1]
        h1.record(stream)
        torch.cuda.synchronize()
        ms2 = h0.elapsed_time(h1) / 2
        also = {"prec": args.also_prec, "value": tqr.nominal_flops(m, n) / (ms2 * 1e-3) / 1e12, "unit": "TFLOP/s",
                "ms_per_step": ms2, "refinement_iterations": it2, "ls_optimality": optimality(X)}
        del ws2
        torch.cuda.empty_cache()

    trees = None
    if not args.no_trees and world == 1:
        # the six trees of the 32768 x 4096 FP64 workload (PlasmaTree with BS = 4) on the
        # same input, and their TS forms (TSQRT / TSMQR for the rows that never pivot)
        trees = {}
        Af = torch.empty_like(A.t()).t()
        T64 = torch.empty(tqr.workspace_size(m, n, 256, 32, "fp64"), dtype=torch.uint8, device=dev)
        tqr.set_timing(True)
        for tr in ("flat", "plasma", "binary", "fibonacci", "greedy", "grasap",
                   "flat-ts", "plasma-ts", "greedy-ts"):
            Af.copy_(A)
            tqr.kernel_time("factor", reset=True)
            tqr.factor(Af, 256, 32, tr, 4, "fp64", T=T64)
            fms = tqr.kernel_time("factor", reset=True)[0]
            cp = tqr.elimlist(-(-m // 256), -(-n // 256), tr, 4)[1]
            trees[tr] = {"factor_ms": fms, "tflops": tqr.nominal_flops(m, n) / (fms * 1e-3) / 1e12, "cp_units": cp}
        tqr.set_timing(False)
        del Af, T64
        torch.cuda.empty_cache()

    batched = None
    if not args.no_batched:
        batched = batched_measurement(args, hbm_peak(), rank, world, dev)
        if args.batch_tensor_prec:
            # the same FP32 batch with tensor-core updates (nb 128; ib and tree autotuned per class)
            tb = batched_measurement(args, hbm_peak(), rank, world, dev, prec=args.batch_tensor_prec)
            batched["tensor_core"] = {k: tb[k] for k in ("value", "unit", "ms_graph_launch", "ms_one_launch_per_matrix",
                                                          "speedup_vs_per_matrix", "tasks", "tuning", "table")}
            batched["tensor_core"]["prec"] = args.batch_tensor_prec
    c5 = c5_measurement(args) if (not args.no_c5 and world == 1) else None
    z64 = z64_measurement(fp64_peak=max(tqr.fp64_peak().values())) if world == 1 else None
    c1 = c1_measurement() if world == 1 else None

    # ---- end to end: host buffers, copies inside the timed region ----
    A_host = A.t().contiguous().cpu().pin_memory()   # (n, m) row-major == A column-major
    b_host = b.t().contiguous().cpu().pin_memory()
    A_dev = torch.empty((n, m), dtype=torch.float64, device=dev)
    b_dev = torch.empty((1, m), dtype=torch.float64, device=dev)
    X_host = torch.empty((1, n), dtype=torch.float64).pin_memory()

    def step_e2e():
        A_dev.copy_(A_host, non_blocking=True)
        b_dev.copy_(b_host, non_blocking=True)
        tqr.lstsq(A_dev.t(), b_dev.t(), 128, 32, args.tree, args.bs, args.prec, tol=tol, max_iter=1000, X=X,
                  workspace=ws, stream=stream)
        X_host.copy_(X.t(), non_blocking=True)

    step_e2e()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        step_e2e()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / args.steps

    step_ms, e2e_ms = replicas.max_over_ranks([ms_total / args.steps, e2e_ms], dev)
    flops = tqr.nominal_flops(m, n)
    value = flops * world / (step_ms * 1e-3) / 1e12
    fac_ms, fac_n = kt["factor"]
    fac_avg = fac_ms / max(fac_n, 1)
    bf16_burst, bf16_sust, peak_src = peaks()
    fp64_pk = tqr.fp64_peak(stream)
    fp64_peak = max(fp64_pk["dfma"], fp64_pk["dmma"])
    achieved = flops / (fac_avg * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"f32 storage, {args.prec} tensor-core updates, FP64 norms/tau/refinement",
        "data": "synthetic", "config": workload_config(args),
        "e2e": {"value": flops * world / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": m * n * 8 + m * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches,
        "roofline": {"kernel": "executor_kernel<float,float,1> (mixed tiled-QR task graph, one launch per step)",
                     "bound": "tensor", "achieved": achieved, "peak": bf16_sust, "unit": "TFLOP/s",
                     "frac": achieved / bf16_sust, "traffic": flops * MIXED_TRAFFIC_PER_FLOP,
                     "traffic_note": "bytes per launch, ncu capture at 24576x2048 (PlasmaTree-TS(16)) scaled "
                                     "by nominal flops",
                     "algorithmic_bytes": tile_task_bytes(args),
                     "algorithmic_bytes_note": "tile-task traffic: C tiles read and written by every task that "
                                               "updates them, split operand images written once and read by "
                                               "every update (no reuse in L2 assumed); A alone is 8mn bytes",
                     "peak_source": f"{peak_src} bf16 dense sustained (MEASURED_PEAKS.json)",
                     "flops_per_launch": flops, "avg_launch_ms": fac_avg,
                     "minimal_bytes": minimal_bytes(args),
                     "minimal_bytes_note": "A (FP32) read and written once plus the T factors (2 p q ib nb "
                                           "FP32) - the least traffic any tiled QR of this shape needs",
                     "traffic_over_minimal": flops * MIXED_TRAFFIC_PER_FLOP / minimal_bytes(args),
                     "traffic_over_tile_task": flops * MIXED_TRAFFIC_PER_FLOP / tile_task_bytes(args),
                     "tensor_issued": tensor_issued(args, fac_avg, bf16_sust)},
        "ls_optimality": {"mixed": eta_mixed, "fp64": eta64, "target": tol},
        "refinement_iterations": iters,
        "fp64": {"value": flops / (fp64_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": fp64_ms,
                 "steps": args.fp64_steps,
                 "frac_of_fp64_peak": flops / (fp64_ms * 1e-3) / 1e12 / fp64_peak,
                 "fp64_peak": {"dfma_tflops": fp64_pk["dfma"], "dmma_tflops": fp64_pk["dmma"],
                               "used": fp64_peak, "nominal": FP64_NOMINAL_TFLOPS,
                               "source": "measured on this GPU by tqr_fp64_peak (DFMA chains on every "
                                         "SM; DMMA m8n8k4 f64 accumulators on every warp)"}},
        "speedup_vs_fp64": fp64_ms / step_ms,
        "also": also,
        "fp64_trees": trees,
        "batched": batched,
        "c5": c5,
        "c1": c1,
        "z64": z64,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "schedule": schedule_bound(args, fac_avg),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line))
    replicas.finalize()


def tensor_issued(args, launch_ms, peak):
    """The MMA work the tensor-core update tasks issue per factorization: 2 (UNMQR) or 3
    (TTMQR / TSMQR) 128 x 128 x 128 products per task, each made of 1 (bf16, fp16), 3
    (split x3) or 6 (split x6) part products - the tensor pipe's load, as against the
    nominal flops, which count the method's arithmetic once."""
    import paper_1303_3182_gb300 as tqr
    parts = {"bf16": 1, "fp16": 1, "bf16x3": 3, "bf16x6": 6}[args.prec]
    c = tqr.plan_counts(args.m, args.n, 128, args.tree, args.bs)
    f = (2 * c["UNMQR"] + 3 * (c["TTMQR"] + c["TSMQR"])) * parts * 2.0 * 128 ** 3
    tf = f / (launch_ms * 1e-3) / 1e12
    return {"flops_per_launch": f, "achieved": tf, "frac": tf / peak, "unit": "TFLOP/s",
            "note": "MMA flops issued by the update tasks (products x part products) per executor launch"}


def minimal_bytes(args, nb=128, ib=32, esz=4):
    """A read and written once plus the T factors: 2 m n esz + 2 p q ib nb esz bytes."""
    p, q = -(-args.m // nb), -(-args.n // nb)
    return 2 * args.m * args.n * esz + 2 * p * q * ib * nb * esz


def tile_task_bytes(args):
    """Algorithmic bytes of one tensor-core factorization as a tile-task graph (nb 128, FP32
    tiles of 64 KB, split operand images of nparts x 32 KB, T blocks of 16 KB): every update
    reads and writes its C tile(s) and reads its operand images (UNMQR: V, Z; TTMQR / TSMQR:
    V2, Z2, T^T); a panel task reads and writes what it factors (GEQRT one tile, TTQRT two
    triangles, TSQRT a triangle and a tile) and writes T; a preparation task reads the
    factored tile and T and writes the images (2 after GEQRT, 3 after TTQRT / TSQRT).  A
    tile touched by consecutive tasks is counted each time: this is the traffic of the
    method when no tile stays in L2 between tasks."""
    import paper_1303_3182_gb300 as tqr
    nparts = {"bf16": 1, "fp16": 1, "bf16x3": 2, "bf16x6": 3}[args.prec]
    tile, img, tblk = 128 * 128 * 4, nparts * 128 * 128 * 2, 32 * 128 * 4
    c = tqr.plan_counts(args.m, args.n, 128, args.tree, args.bs)
    panel = c["GEQRT"] * (2 * tile + tblk) + c["TTQRT"] * (2 * tile + tblk) + c["TSQRT"] * (3 * tile + tblk)
    prep = c["GEQRT"] * (tile + tblk + 2 * img) + (c["TTQRT"] + c["TSQRT"]) * (tile + tblk + 3 * img)
    upd = c["UNMQR"] * (2 * tile + 2 * img) + (c["TTMQR"] + c["TSMQR"]) * (4 * tile + 3 * img)
    return panel + prep + upd


def schedule_bound(args, executor_ms):
    """The executor's span against the thesis's Chapter 5 bounds for its task graph on
    the GPU's resident CTAs, with the measured mean task durations as weights: the
    CP-method list schedule (the default claim order of the tensor-core path) and the
    ALAP Derived Performance Bound."""
    import torch

    import paper_1303_3182_gb300 as tqr
    nproc = torch.cuda.get_device_properties(0).multi_processor_count
    p, q = -(-args.m // 128), -(-args.n // 128)
    ms, bound, lost = tqr.schedule(p, q, args.tree, args.bs, nproc, TENSOR_TASK_MEAN_US)
    return {"claim_order": "CP-method list schedule on the resident CTAs (library default for tensor-core "
                           "precisions)", "claim_weights": list(TENSOR_CLAIM_WEIGHTS), "processors": nproc,
            "task_mean_us": list(TENSOR_TASK_MEAN_US),
            "list_schedule_ms": ms / 1e3, "alap_bound_ms": bound / 1e3, "executor_ms": executor_ms,
            "executor_over_alap_bound": executor_ms / (bound / 1e3),
            "note": "list schedule and ALAP Derived bound of the task graph with the measured mean task "
                    "durations as weights"}


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    main_gpu(args)


if __name__ == "__main__":
    main()
