"""Pins for the bounded-processor scheduling oracle (thesis Chapter 5): the CP-method
list schedule and the ALAP Derived Performance Bound on the tiled-QR task graph.

Expected values are printed in the thesis (tests/golden/schedule_5x5.txt, citing its
table) or follow from classical scheduling facts (a list schedule on one processor runs
every task back to back; with as many processors as tasks it is the as-soon-as-possible
schedule; Graham's bound; the ALAP bound is a lower bound of every schedule).
"""
import os

import pytest

from oracle import elimlists as E
from oracle import schedule as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "schedule_5x5.txt")
COLS = {"grasap": 3, "greedy": 4, "fibonacci": 5, "flat": 6}
TREES = {"grasap": E.GRASAP, "greedy": E.GREEDY, "fibonacci": E.FIBONACCI, "flat": E.FLAT}


def _rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def _graph(p, q, tree, weights=S.DEFAULT_WEIGHTS):
    return S.task_graph(p, q, E.elimination_list(p, q, tree, bs=2), weights)


@pytest.mark.parametrize("tree", sorted(COLS))
def test_cp_method_5x5_table(tree):
    g = _graph(5, 5, TREES[tree])
    checked = 0
    for row in _rows():
        cell = row[COLS[tree]]
        if cell.endswith("*"):
            continue
        assert S.list_schedule(g, int(row[0]))[0] == int(cell), (tree, row[0])
        checked += 1
    assert checked >= 12


def test_alap_bound_5x5_table():
    g = _graph(5, 5, E.GRASAP)
    for row in _rows():
        assert S.alap_bound(g, int(row[0]))[0] == int(row[1]), row[0]


def test_sequential_work_and_critical_path_agree_with_chapter3():
    """The explicit graph has the thesis's total work 6pq^2 - 2q^3 (p >= q) and the
    critical path of the independent earliest-finish simulation of oracle.elimlists."""
    for p, q in [(5, 5), (15, 6), (8, 3), (4, 7)]:
        for tree in TREES.values():
            elims = E.elimination_list(p, q, tree)
            g = S.task_graph(p, q, elims)
            if p >= q:
                assert sum(g.weight) == 6 * p * q * q - 2 * q ** 3
            assert S.critical_path(g) == E.critical_path(p, q, elims)


@pytest.mark.parametrize("p,q", [(5, 5), (12, 4), (7, 7), (20, 3)])
def test_list_schedule_extremes_and_graham_bound(p, q):
    for tree in TREES.values():
        g = _graph(p, q, tree)
        tseq, cp = sum(g.weight), S.critical_path(g)
        assert S.list_schedule(g, 1)[0] == tseq
        assert S.list_schedule(g, len(g))[0] == cp
        for nproc in (2, 3, 5, 8, 13):
            ms, start = S.list_schedule(g, nproc)
            # every task starts after all its predecessors finished
            for t in range(len(g)):
                for d in g.preds[t]:
                    assert start[t] >= start[d] + g.weight[d]
            # never more than nproc tasks at once
            ev = sorted([(start[t], 1) for t in range(len(g))] +
                        [(start[t] + g.weight[t], -1) for t in range(len(g))], key=lambda x: (x[0], x[1]))
            run = 0
            for _, d in ev:
                run += d
                assert run <= nproc
            # Graham: a list schedule is within T_seq / P + (1 - 1/P) CP
            assert ms * nproc <= tseq + (nproc - 1) * cp
            # the ALAP Derived bound never exceeds a schedule's length
            assert S.alap_bound(g, nproc)[0] <= ms


def test_alap_bound_limits():
    g = _graph(15, 6, E.GREEDY)
    tseq, cp = sum(g.weight), S.critical_path(g)
    assert S.alap_bound(g, 1) == (tseq, 0)
    assert S.alap_bound(g, len(g))[0] == cp


def _tiled_cholesky(t):
    """Task graph of the right-looking tiled Cholesky factorization of t x t tiles (one region
    per tile), weights POTRF 1, TRSM 3, SYRK 3, GEMM 6: the thesis's own example for the ALAP
    Derived bound (the procedure is the same for any task graph)."""
    g = S.TaskGraph()
    for k in range(t):
        g.add(0, ("POTRF", k), 1, [], [(k, k)])
        for i in range(k + 1, t):
            g.add(1, ("TRSM", i, k), 3, [(k, k)], [(i, k)])
        for i in range(k + 1, t):
            g.add(2, ("SYRK", i, k), 3, [(i, k)], [(i, i)])
            for j in range(k + 1, i):
                g.add(3, ("GEMM", i, j, k), 6, [(i, k), (j, k)], [(i, j)])
    return g


def test_alap_lost_area_cholesky_5x5_figure_and_table():
    """The lost areas of the ALAP execution (walking back until more than p tasks are
    active) and the unrounded bound (T_seq + LA_p) / p of the thesis's 5 x 5 Cholesky example."""
    g = _tiled_cholesky(5)
    tseq, cp = sum(g.weight), S.critical_path(g)
    assert (tseq, cp) == (125, 35)
    path = os.path.join(os.path.dirname(__file__), "golden", "alap_cholesky_5x5.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    for procs, la, tp in rows:
        p = int(procs)
        _, lost = S.alap_bound(g, p)
        if la != "-":
            assert lost == int(la), p
        assert round(max(cp, (tseq + lost) / p), 2) == float(tp), p
