"""Run and time one path of the library on seeded inputs (for timing runs and profilers).

    python -m paper_1303_3182_gb300.profile --m 4096 --n 1024 --prec bf16x3 --reps 3 \
        [--trace trace.json]
    python -m paper_1303_3182_gb300.profile --batch 256 --prec fp32 --reps 3
    python -m paper_1303_3182_gb300.profile --lstsq --m 16384 --n 4096 --prec bf16x6 --reps 2

Default mode: tqr_factor of an N(0,1) matrix; one JSON line per repetition (device time
of the factorization executor and the nominal TFLOP/s).  With --trace, the last
repetition records the executor's per-task stamps (tqr_set_trace) and writes them as a
list of {kind, i, piv, k, j, sm, start_us, end_us, phases_us} records - a Gantt chart of
the task graph.  phases_us: four time slots of the task - panel tasks: panel, T, in-tile
trailing update (summed over ib-blocks) and the resident tiles' loads; tensor-core updates:
the first product with its operand images, its wait, the second product(s), the epilogue;
operand preparation: loads, Gram matrix and T_full, Z = V T_full^T, the split images.
--batch N: one batched launch (tqr_batch_plan_run, built-in size classes) over the
first N matrices of the 2048-matrix distribution (rows uniform in [256, 8192], columns
in {32, 64, 128, 256}).
--lstsq: tqr_lstsq of A = U diag(sigma) V^T (cond --cond) with one right-hand side
b = A x + 1e-3 N(0,1); reports the kernel time of factorization and refinement.
"""
from __future__ import annotations

import argparse
import json


def _factor(a, tqr, torch):
    nb = a.nb or (256 if a.prec == "fp64" else 128)
    dt = torch.float64 if a.prec == "fp64" else torch.float32
    g = torch.Generator(device="cuda")
    g.manual_seed(a.seed)
    A0 = torch.randn(a.n, a.m, dtype=torch.float64, device="cuda", generator=g).to(dt).t()
    work = torch.empty_like(A0.t()).t()
    T = torch.empty(tqr.workspace_size(a.m, a.n, nb, a.ib, a.prec), dtype=torch.uint8, device="cuda")
    tqr.set_timing(True)
    for r in range(a.reps):
        work.copy_(A0)
        last = r == a.reps - 1
        if last and a.trace:
            tqr.set_trace(True)
        tqr.kernel_time("factor", reset=True)
        tqr.factor(work, nb, a.ib, a.tree, a.bs, a.prec, T=T)
        ms, _ = tqr.kernel_time("factor", reset=True)
        print(json.dumps({"rep": r, "m": a.m, "n": a.n, "nb": nb, "ib": a.ib, "prec": a.prec, "tree": a.tree,
                          "ms": ms, "tflops": tqr.nominal_flops(a.m, a.n) / (ms * 1e-3) / 1e12}), flush=True)
    if a.trace:
        tqr.set_trace(False)
        tr = tqr.trace_fetch()
        t0 = int(tr[:, 4].min())
        names = ["GEQRT", "TTQRT", "UNMQR", "TTMQR", "UNMQR_B", "TTMQR_B", "TSQRT", "TSMQR", "TSMQR_B",
                 "PREP_G", "PREP_T", "TTQRT_S", "TSQRT_S"]
        recs = [{"kind": names[int(r[0])], "i": int(r[1]), "piv": int(r[2]), "k": int(r[3]) & 0xFFFF,
                 "j": (int(r[3]) >> 16) if (int(r[3]) >> 16) < 32768 else -1, "sm": int(r[7]),
                 "start_us": (int(r[5]) - t0) / 1e3, "end_us": (int(r[6]) - t0) / 1e3,
                 "phases_us": [int(x) / 1e3 for x in r[8:12]]} for r in tr]
        with open(a.trace, "w") as f:
            json.dump(recs, f)


def _batch(a, tqr, torch):
    import synthetic
    from .autotune import DeviceBatch, time_launch
    shapes = synthetic.ragged_batch_shapes(2048, seed=synthetic.SEED_BASE + 4)[:a.batch]
    db = DeviceBatch(shapes, synthetic.SEED_BASE + 4, dtype=torch.float64 if a.prec == "fp64" else torch.float32)
    plan = tqr.BatchPlan(db.As, a.prec)
    flops = plan.info()["flops"]
    for r in range(a.reps):
        ms = time_launch(plan, db.restore, reps=1, use_graph=True)
        print(json.dumps({"rep": r, "batch": a.batch, "prec": a.prec, "tasks": plan.info()["tasks"], "ms": ms,
                          "tflops": flops / (ms * 1e-3) / 1e12}), flush=True)
    plan.close()


def _lstsq(a, tqr, torch):
    import synthetic
    nb = a.nb or (256 if a.prec == "fp64" else 128)
    A, _, b = synthetic.least_squares_device(a.m, a.n, a.cond, 1e-3, 1, synthetic.SEED_BASE + 3, torch.device("cuda"))
    ws = torch.empty(tqr.lstsq_workspace_size(a.m, a.n, 1, nb, a.ib, a.prec), dtype=torch.uint8, device="cuda")
    X = tqr.colmajor(torch.empty((a.n, 1), dtype=torch.float64, device="cuda"))
    tqr.set_timing(True)
    for r in range(a.reps):
        for k in ("factor", "refine"):
            tqr.kernel_time(k, reset=True)
        _, it = tqr.lstsq(A, b, nb, a.ib, a.tree, a.bs, a.prec, tol=1e-14, max_iter=1000, X=X, workspace=ws,
                          return_iters=True)
        kt = {k: tqr.kernel_time(k, reset=True)[0] for k in ("factor", "refine")}
        print(json.dumps({"rep": r, "m": a.m, "n": a.n, "prec": a.prec, "iters": it, "kernel_ms": kt}), flush=True)


def main():
    import torch

    import paper_1303_3182_gb300 as tqr
    from paper_1303_3182_gb300 import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--nb", type=int, default=0, help="0: 128 for tensor-core precisions, 256 for fp64")
    ap.add_argument("--ib", type=int, default=32)
    ap.add_argument("--tree", default="greedy")
    ap.add_argument("--bs", type=int, default=4)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1303318202)
    ap.add_argument("--trace", default="")
    ap.add_argument("--order", type=int, default=0,
                    help="executor claim order: 0 = earliest start (unbounded processors), 1 = bounded CP method")
    ap.add_argument("--weights", default="", help="claim-order kernel weights GEQRT,TTQRT,UNMQR,TTMQR (--order 1)")
    ap.add_argument("--batch", type=int, default=0, help="batched mode: number of matrices")
    ap.add_argument("--lstsq", action="store_true", help="least-squares mode")
    ap.add_argument("--cond", type=float, default=1e6)
    a = ap.parse_args()
    build.build()
    if a.order:
        tqr.set_claim_order(a.order, [int(x) for x in a.weights.split(",")] if a.weights else None)
    if a.batch:
        _batch(a, tqr, torch)
    elif a.lstsq:
        _lstsq(a, tqr, torch)
    else:
        _factor(a, tqr, torch)


if __name__ == "__main__":
    main()
