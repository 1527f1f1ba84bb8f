"""Per-size-class autotuner of the batched factorization (tqr_batch_plan_*).

Matrices are grouped into size classes (a row-count bucket x an exact column count);
for each class a sample of its matrices is factored as one batched launch under
candidate (nb, ib, tree) settings, in three stages: the tile size nb (Greedy, ib 32),
then the inner block ib at the best nb, then the elimination tree at the best (nb, ib).
The result is a tuning table (rows m_lo, m_hi, n_lo, n_hi, nb, ib, tree, bs) for
tqr_batch_params.  All timing is device time (CUDA events around one graph-replayed
launch, inputs restored between launches).

    python -m paper_1303_3182_gb300.autotune --count 2048 --prec fp32 --out table.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import BatchPlan, TREES, batch_params

M_BUCKETS = ((1, 1024), (1025, 4096), (4097, 1 << 40))
NB_CANDIDATES = (32, 64, 128, 256)
IB_CANDIDATES = (8, 16, 32)
TREE_CANDIDATES = (("greedy", 1), ("binary", 1), ("fibonacci", 1), ("flat", 1), ("plasma", 4))


def size_classes(shapes, m_buckets=M_BUCKETS):
    """{(m_lo, m_hi, n): [matrix indices]} over the given shapes."""
    out = {}
    for b, (m, n) in enumerate(shapes):
        for lo, hi in m_buckets:
            if lo <= m <= hi:
                out.setdefault((lo, hi, int(n)), []).append(b)
                break
    return out


class DeviceBatch:
    """All matrices of a batch in one device buffer (column-major views) plus a pristine
    copy to restore the inputs between timed launches."""

    def __init__(self, shapes, seed, device="cuda", dtype=None):
        import torch
        dtype = dtype or torch.float32
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        sizes = [m * n for m, n in self.shapes]
        # 16-byte aligned starts so that vector loads stay allowed
        self.offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
        for b, s in enumerate(sizes):
            self.offsets[b + 1] = self.offsets[b] + (s + 3) // 4 * 4
        total = int(self.offsets[-1])
        self.buf = torch.empty(total, dtype=dtype, device=device)
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        self.buf.normal_(generator=g)
        self.src = self.buf.clone()
        self.As = [self.buf[int(o):int(o) + m * n].view(n, m).t()
                   for o, (m, n) in zip(self.offsets[:-1], self.shapes)]

    def restore(self):
        self.buf.copy_(self.src)

    def subset(self, idx):
        return [self.As[b] for b in idx]

    @property
    def bytes(self):
        return self.buf.numel() * self.buf.element_size()


def time_launch(plan, restore, reps=3, use_graph=True):
    """Median device ms of one plan launch (inputs restored, untimed, before each)."""
    import torch
    from . import set_sync
    stream = torch.cuda.current_stream()
    restore()
    plan.run(use_graph=use_graph)
    ts = []
    old = set_sync(False)
    try:
        for _ in range(reps):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(use_graph=use_graph)
            e1.record(stream)
            plan.status()
            ts.append(e0.elapsed_time(e1))
    finally:
        set_sync(old)
    return float(np.median(ts))


def _time_params(db, idx, prec, params, reps):
    As = db.subset(idx)
    plan = BatchPlan(As, prec, params=np.asarray(params, dtype=np.int32).reshape(-1, 4))
    try:
        return time_launch(plan, db.restore, reps=reps)
    finally:
        plan.close()


def autotune(shapes, prec="fp32", seed=1303318204, reps=3, per_class=128, device="cuda", log=None):
    """Tuning table rows and a per-class report for the given shapes."""
    tensor = prec not in ("fp32", "fp64")
    import torch
    db = DeviceBatch(shapes, seed, device, torch.float64 if prec == "fp64" else torch.float32)
    rows, report = [], []
    for (lo, hi, n), idx in sorted(size_classes(shapes).items()):
        idx = idx[:per_class]
        m_max = max(db.shapes[b][0] for b in idx)
        tried = {}

        def run(nb, ib, tree, bs):
            key = (nb, ib, tree, bs)
            if key not in tried:
                params = [[nb, ib, TREES[tree], bs]] * len(idx)
                tried[key] = _time_params(db, idx, prec, params, reps)
                if log:
                    log(f"class m {lo}..{hi} n {n}: nb {nb} ib {ib} {tree}/{bs}: {tried[key]:.3f} ms")
            return tried[key]

        if tensor:
            nb, ib = 128, 32
        else:
            nbs = [c for c in NB_CANDIDATES if c <= max(32, m_max)]
            nb = min(nbs, key=lambda c: run(c, min(c, 32), "greedy", 1))
            ib = min([c for c in IB_CANDIDATES if c <= nb], key=lambda c: run(nb, c, "greedy", 1))
        tree, bs = min(TREE_CANDIDATES, key=lambda t: run(nb, ib, t[0], t[1]))
        best = tried[(nb, ib, tree, bs)]
        default = batch_params([db.shapes[b][0] for b in idx], [n] * len(idx), prec)[0]
        rows.append([lo, hi, n, n, nb, ib, TREES[tree], bs])
        report.append({"m": [lo, hi], "n": n, "matrices": len(idx), "nb": nb, "ib": ib, "tree": tree, "bs": bs,
                       "ms": best, "builtin": [int(x) for x in default],
                       "tried": {f"{k[0]}/{k[1]}/{k[2]}/{k[3]}": v for k, v in tried.items()}})
    return rows, report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=1303318204)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--per-class", type=int, default=128)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    import synthetic
    from . import build
    build.build()
    shapes = synthetic.ragged_batch_shapes(args.count, seed=args.seed)
    t0 = time.time()
    rows, report = autotune(shapes, args.prec, args.seed, args.reps, args.per_class, log=print)
    doc = {"prec": args.prec, "table": rows, "classes": report, "seconds": time.time() - t0}
    text = json.dumps(doc, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
