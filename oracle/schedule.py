"""Bounded-processor scheduling of the tiled-QR task graph (thesis Chapter 5).

Test infrastructure only: the CPU oracle for the library's bounded-processor schedule.
Only the tests use it; the library never imports it and it imports nothing from the
library.

Contents
--------
* ``task_graph(p, q, elims)``: the explicit task graph of an elimination list -- the
  column-by-column sequential program of Algorithm "elimTR" (Section 3.1.1), each task
  depending on the last writer of every tile region it reads or writes and on the
  readers since that write of every region it writes (the precedences of Eq. (ttdeps)
  and (ttdeps2); the regions are each tile's strictly lower part 'L' and upper part 'U').
* ``bottom_levels``: the Backflow priorities of Section "Critical Path Scheduling" --
  a task's priority is its processing time plus the largest priority of its successors.
* ``list_schedule(graph, nproc)``: the "CP Method" -- at every moment the free
  processors take, among the tasks whose predecessors have all finished, those of
  largest priority; the result is the makespan and every task's start time.
* ``alap_bound(graph, nproc)``: the ALAP Derived Performance Bound of Eq. (alapbound):
  every task starts as late as possible on unbounded processors; walking back from the
  end of that execution, LA_p accumulates the idle area of p processors until the first
  moment at which more than p tasks are active; the bound on the makespan is
  max(critical path, ceil((T_seq + LA_p) / p)) (makespans of integer weights are
  integers, so the bound is rounded up).

Readings (the section defines the procedures in words only): ties between tasks of equal
priority go to the task that comes first in the sequential program; the backward walk of
the lost area stops where more than p processors are needed ("more processors needed to
keep the critical path length constant").  With these, the CP-method makespans and the
ALAP Derived bounds of Table "Schedule lengths for matrix of 5x5 tiles" are reproduced
except three cells (see tests/golden/schedule_5x5.txt), and the lost areas of the thesis's
own 5 x 5 tiled Cholesky example (Figure "ALAP execution for 5 x 5 tiles": 0, 4, 11, 24, 45
for 1..5 processors; stopping at "p or more active tasks" would give 40 for 5) with the
unrounded bounds of its Table "Upper bound on speedup and efficiency for 5x5 tiles".
"""
from __future__ import annotations

import heapq

from .elimlists import W_GEQRT, W_TTMQR, W_TTQRT, W_UNMQR

GEQRT, TTQRT, UNMQR, TTMQR = range(4)
DEFAULT_WEIGHTS = (W_GEQRT, W_TTQRT, W_UNMQR, W_TTMQR)


class TaskGraph:
    """Tasks in sequential-program order (a topological order) with their kind, tile
    coordinates, weight and predecessor / successor lists."""

    def __init__(self):
        self.kind, self.key, self.weight = [], [], []
        self.preds, self.succs = [], []
        self._last_writer = {}   # region -> task index
        self._readers = {}       # region -> task indices that read it since its last write

    def add(self, kind, key, weight, reads, writes):
        t = len(self.kind)
        deps = set()
        for r in list(reads) + list(writes):
            if r in self._last_writer:
                deps.add(self._last_writer[r])
        for r in writes:
            deps.update(self._readers.get(r, ()))
        deps.discard(t)
        for r in reads:
            self._readers.setdefault(r, set()).add(t)
        for r in writes:
            self._last_writer[r] = t
            self._readers[r] = set()
        self.kind.append(kind)
        self.key.append(key)
        self.weight.append(weight)
        self.preds.append(sorted(deps))
        self.succs.append([])
        for d in deps:
            self.succs[d].append(t)
        return t

    def __len__(self):
        return len(self.kind)


def task_graph(p: int, q: int, elims, weights=DEFAULT_WEIGHTS) -> TaskGraph:
    """Explicit task graph of the TT tiled QR driven by an elimination list of triples
    (k, i, piv), 0-based; weights are per kind (GEQRT, TTQRT, UNMQR, TTMQR)."""
    g = TaskGraph()
    by_col = {}
    for e in elims:
        by_col.setdefault(e[0], []).append(e)
    for k in range(min(p, q)):
        for i in range(k, p):
            g.add(GEQRT, (i, k), weights[GEQRT], [], [(i, k, "L"), (i, k, "U")])
            for j in range(k + 1, q):
                g.add(UNMQR, (i, k, j), weights[UNMQR], [(i, k, "L")], [(i, j, "L"), (i, j, "U")])
        for (_, i, piv) in by_col.get(k, []):
            g.add(TTQRT, (i, piv, k), weights[TTQRT], [], [(piv, k, "U"), (i, k, "U")])
            for j in range(k + 1, q):
                g.add(TTMQR, (i, piv, k, j), weights[TTMQR], [(i, k, "U")],
                      [(piv, j, "L"), (piv, j, "U"), (i, j, "L"), (i, j, "U")])
    return g


def bottom_levels(g: TaskGraph):
    """Backflow priorities: cp(t) = weight(t) + max over successors s of cp(s)."""
    n = len(g)
    cp = [0] * n
    for t in range(n - 1, -1, -1):
        cp[t] = g.weight[t] + max((cp[s] for s in g.succs[t]), default=0)
    return cp


def critical_path(g: TaskGraph) -> int:
    return max(bottom_levels(g), default=0)


def list_schedule(g: TaskGraph, nproc: int):
    """CP Method on nproc processors.  Event-driven: at time t every finished task
    releases its successors; then, while a processor is free, the ready task of largest
    priority starts (ties: earlier in the sequential program).  Returns (makespan,
    start times)."""
    n = len(g)
    cp = bottom_levels(g)
    missing = [len(g.preds[t]) for t in range(n)]
    ready = [(-cp[t], t) for t in range(n) if missing[t] == 0]
    heapq.heapify(ready)
    running = []           # (finish time, task)
    start = [None] * n
    free, now, done = nproc, 0, 0
    while done < n:
        while free > 0 and ready:
            _, t = heapq.heappop(ready)
            start[t] = now
            heapq.heappush(running, (now + g.weight[t], t))
            free -= 1
        now = running[0][0]
        while running and running[0][0] == now:
            _, t = heapq.heappop(running)
            free += 1
            done += 1
            for s in g.succs[t]:
                missing[s] -= 1
                if missing[s] == 0:
                    heapq.heappush(ready, (-cp[s], s))
    makespan = max((start[t] + g.weight[t] for t in range(n)), default=0)
    return makespan, start


def alap_bound(g: TaskGraph, nproc: int):
    """ALAP Derived Performance Bound for nproc processors: returns (bound, LA_p), the
    bound being max(CP, ceil((T_seq + LA_p) / nproc))."""
    cp = bottom_levels(g)
    crit = max(cp, default=0)
    tseq = sum(g.weight)
    # active-task count of the ALAP execution (task t runs over [crit - cp[t], crit - cp[t] + w))
    events = {}
    for t in range(len(g)):
        s = crit - cp[t]
        events[s] = events.get(s, 0) + 1
        events[s + g.weight[t]] = events.get(s + g.weight[t], 0) - 1
    times = sorted(events)
    segs = []            # (t0, t1, active)
    active = 0
    for a, b in zip(times, times[1:]):
        active += events[a]
        segs.append((a, b, active))
    lost = 0
    for (a, b, act) in reversed(segs):
        if act > nproc:
            break
        lost += (nproc - act) * (b - a)
    return max(crit, -(-(tseq + lost) // nproc)), lost
