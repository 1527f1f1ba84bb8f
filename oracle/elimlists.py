"""Elimination lists, the tile task graph and its critical path (thesis Chapter 3).

Test infrastructure only: this module is the CPU oracle for the integer side of tiled
QR.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark use it;
the library never imports it and it imports nothing from the library.

Conventions
-----------
* Rows and columns are 0-based (the thesis counts from 1).
* An elimination is a triple ``(k, i, piv)``: tile ``(i, k)`` is zeroed by a
  triangle-on-triangle transformation with pivot row ``piv`` in panel ``k``
  (the thesis's elim(i, piv(i,k), k), Section 3.1, Algorithm "Generic QR").
* Every generator returns the list in canonical order: by column, then by the
  time step (or level) inside the column, then by row.

Each generator follows the definition in Section 3.2; the task graph follows the
TT elimination of Algorithm "elimTR" read as the column-by-column sequential program
(Section 3.1.1) with the dependencies of Eq. (ttdeps) and (ttdeps2), and kernel
weights GEQRT 4, TTQRT 2, UNMQR 6, TTMQR 6 (Table "Kernels for tiled QR").
"""
from __future__ import annotations

FLAT, PLASMA, BINARY, FIBONACCI, GREEDY, GRASAP, ASAP = range(7)
TREE_NAMES = {FLAT: "flat", PLASMA: "plasma", BINARY: "binary", FIBONACCI: "fibonacci",
              GREEDY: "greedy", GRASAP: "grasap", ASAP: "asap"}

W_GEQRT, W_TTQRT, W_UNMQR, W_TTMQR = 4, 2, 6, 6
# TS (triangle on top of square) kernels, Table "Kernels for tiled QR"
W_TSQRT, W_TSMQR = 6, 12


def _v2(d: int) -> int:
    """Number of trailing zero bits of d >= 1."""
    n = 0
    while d % 2 == 0:
        d //= 2
        n += 1
    return n


# ---------------------------------------------------------------------------
# Generators (Section 3.2.1 coarse-grain schemes, Section 3.2.4 PlasmaTree)
# ---------------------------------------------------------------------------

def flat_tree(p: int, q: int):
    """Sameh-Kuck / FlatTree: every tile of column k is zeroed by the diagonal row k,
    top to bottom (Section 3.2.1, 'Sameh-Kuck algorithm')."""
    out = []
    for k in range(min(p, q)):
        for i in range(k + 1, p):
            out.append((k, i, k))
    return out


def fibonacci_coarse(p: int, q: int):
    """Modi-Clarke Fibonacci scheme of order 1 (Section 3.2.1).

    Returns (list, coarse) where coarse[(i, k)] is the time step at which tile (i, k)
    is zeroed.  First column (thesis numbering, rows r = 2..p): x is the least integer
    with x(x+1)/2 >= p-1 and coarse(r,1) = x - y + 1, y the least integer with
    r <= y(y+1)/2 + 1.  Column k is column 1 shifted down k-1 rows plus 2(k-1) steps.
    A run of z consecutive rows zeroed at the same step uses the z rows right above
    it, in order; z counts only rows that exist (the bottom run is cut at row p).
    """
    x = 0
    while x * (x + 1) // 2 < p - 1:
        x += 1

    def coarse1(r):  # r: thesis row index >= 2 of column 1
        y = 0
        while r > y * (y + 1) // 2 + 1:
            y += 1
        return x - y + 1

    coarse = {}
    out = []
    for k in range(min(p, q)):
        # thesis: column K = k+1, rows I = K+1..p  <->  0-based rows i = k+1..p-1
        steps = {}
        for i in range(k + 1, p):
            r1 = (i + 1) - (k + 1) + 1  # row of column 1 that is shifted onto row i
            s = coarse1(r1) + 2 * k
            coarse[(i, k)] = s
            steps.setdefault(s, []).append(i)
        for s in sorted(steps):
            rows = sorted(steps[s])
            z = len(rows)
            for i in rows:
                out.append((k, i, i - z))
    return out, coarse


def greedy_coarse(p: int, q: int):
    """Greedy (Section 3.2.1; equivalently Algorithm 'tiled-greedy').

    At coarse step s, in every column k the live rows are those not yet zeroed in
    column k and (for k > 0) zeroed in column k-1 at a step <= s-1.  With n live rows,
    the bottom floor(n/2) are zeroed by the floor(n/2) live rows right above them,
    paired in order.  Returns (list, coarse).
    """
    kmax = min(p, q)
    zeroed = {}
    remaining = sum(p - 1 - k for k in range(kmax))
    by_col = [[] for _ in range(kmax)]
    s = 0
    while remaining > 0:
        s += 1
        for k in range(kmax):
            live = [i for i in range(k, p)
                    if (i, k) not in zeroed and (k == 0 or zeroed.get((i, k - 1), s) <= s - 1)]
            n = len(live)
            h = n // 2
            for j in range(h):
                i, piv = live[n - h + j], live[n - 2 * h + j]
                by_col[k].append((s, i, piv))
                zeroed[(i, k)] = s
                remaining -= 1
    out = []
    for k in range(kmax):
        for s_, i, piv in sorted(by_col[k]):
            out.append((k, i, piv))
    return out, zeroed


def binary_tree(p: int, q: int):
    """BinaryTree = PlasmaTree with domain size 1 (Section 3.2.4): in column k, row
    k+d (d >= 1) is zeroed at level v2(d) by row k + d - 2**v2(d)."""
    return plasma_tree(p, q, 1)


def plasma_tree(p: int, q: int, bs: int):
    """PlasmaTree(BS) (Section 3.2.4): in column k, domains of bs consecutive rows start
    at the diagonal row k (the bottom one is cut at row p).  Inside a domain the first
    row zeroes the others top-down (flat); then the domain heads are merged by a binary
    tree (head d is zeroed at level v2(d) by head d - 2**v2(d))."""
    if bs < 1:
        raise ValueError("bs must be >= 1")
    out = []
    for k in range(min(p, q)):
        heads = list(range(k, p, bs))
        for h in heads:
            for i in range(h + 1, min(h + bs, p)):
                out.append((k, i, h))
        merge = []
        for d in range(1, len(heads)):
            lvl = _v2(d)
            merge.append((lvl, d, heads[d], heads[d - (1 << lvl)]))
        for lvl, d, i, piv in sorted(merge):
            out.append((k, i, piv))
    return out


# ---------------------------------------------------------------------------
# Task graph and timing with unbounded processors (Section 3.1.3)
# ---------------------------------------------------------------------------

class TileSchedule:
    """Earliest-finish-time simulation of the tile task graph, built incrementally in
    the order of the sequential program.

    Each tile (i, j) holds two regions: 'L' (strictly lower part: the GEQRT
    reflectors) and 'U' (upper triangle: R, later the TTQRT reflectors).  A task starts
    when every earlier task it conflicts with (read-after-write, write-after-write,
    write-after-read on a region) has finished; it lasts its kernel weight.  This gives
    exactly the precedences of Eq. (ttdeps) and (ttdeps2), and lets UNMQR(i,k,j)
    overlap TTQRT(i,piv,k) because one reads 'L' and the other writes 'U'.
    """

    def __init__(self):
        self.last_write = {}   # region -> finish time of its last writer
        self.read_since = {}   # region -> latest finish of readers since that write
        self.finish = {}       # task key -> finish time
        self.makespan = 0

    def add(self, key, weight, reads, writes):
        start = 0
        for r in reads:
            start = max(start, self.last_write.get(r, 0))
        for r in writes:
            start = max(start, self.last_write.get(r, 0), self.read_since.get(r, 0))
        end = start + weight
        for r in reads:
            self.read_since[r] = max(self.read_since.get(r, 0), end)
        for r in writes:
            self.last_write[r] = end
            self.read_since[r] = 0
        self.finish[key] = end
        self.makespan = max(self.makespan, end)
        return end

    # -- the four kernels ---------------------------------------------------
    def geqrt(self, i, k):
        return self.add(("GEQRT", i, k), W_GEQRT, [], [(i, k, "L"), (i, k, "U")])

    def unmqr(self, i, k, j):
        return self.add(("UNMQR", i, k, j), W_UNMQR, [(i, k, "L")], [(i, j, "L"), (i, j, "U")])

    def ttqrt(self, i, piv, k):
        return self.add(("TTQRT", i, piv, k), W_TTQRT, [], [(piv, k, "U"), (i, k, "U")])

    def ttmqr(self, i, piv, k, j):
        return self.add(("TTMQR", i, piv, k, j), W_TTMQR, [(i, k, "U")],
                        [(piv, j, "L"), (piv, j, "U"), (i, j, "L"), (i, j, "U")])

    def tsqrt(self, i, piv, k):
        # the square tile (i, k) is overwritten as a whole by its reflectors
        return self.add(("TSQRT", i, piv, k), W_TSQRT, [],
                        [(piv, k, "U"), (i, k, "L"), (i, k, "U")])

    def tsmqr(self, i, piv, k, j):
        return self.add(("TSMQR", i, piv, k, j), W_TSMQR, [(i, k, "L"), (i, k, "U")],
                        [(piv, j, "L"), (piv, j, "U"), (i, j, "L"), (i, j, "U")])


def _column_panel(sched: TileSchedule, p, q, k, skip=()):
    """GEQRT(i,k) then UNMQR(i,k,j) for every row i >= k of panel k (except the rows in
    skip, which a TS kernel zeroes while still square)."""
    g = {}
    for i in range(k, p):
        if i in skip:
            continue
        g[i] = sched.geqrt(i, k)
        for j in range(k + 1, q):
            sched.unmqr(i, k, j)
    return g


def _column_elims(sched: TileSchedule, q, k, elims, ts_rows=()):
    for (_, i, piv) in elims:
        if i in ts_rows:
            sched.tsqrt(i, piv, k)
            for j in range(k + 1, q):
                sched.tsmqr(i, piv, k, j)
        else:
            sched.ttqrt(i, piv, k)
            for j in range(k + 1, q):
                sched.ttmqr(i, piv, k, j)


def ts_rows(elims):
    """Rows zeroed by TS kernels in the TS form of a list: {k: set of rows}.

    A TS elimination (Algorithm "elimSQ") zeroes a square tile, so its row must not
    have been triangularized in that column; a pivot always is (GEQRT(piv,k) precedes
    TSQRT).  The TS form of a list therefore zeroes with TSQRT/TSMQR every row that is
    never a pivot in the column (a leaf of the column's tree) and keeps the TT kernels
    for the rows that pivot before they are zeroed.  FlatTree's TS form is Sameh-Kuck
    with TS kernels; PlasmaTree(BS)'s is the PLASMA algorithm (TS inside a domain, TT
    between the domain heads)."""
    piv_rows = {}
    for (k, _, piv) in elims:
        piv_rows.setdefault(k, set()).add(piv)
    out = {}
    for (k, i, _) in elims:
        if i not in piv_rows.get(k, ()):
            out.setdefault(k, set()).add(i)
    return out


def asap_column(p: int, k: int, ready: dict):
    """ASAP on one tile column (Section 3.2.2; Definition 'optiter' with w = 2).

    ready[i] is the finish time of GEQRT(i, k) for rows i >= k.  At each event time t,
    the rows that are triangularised, not zeroed and not busy form the ready set; with
    n >= 2 of them, s = floor(n/2) eliminations start at once: of the bottom 2s ready
    rows r_1 < ... < r_2s, row r_{s+j} is zeroed by r_j (an odd leftover is the top
    ready row).  A pivot is busy until t + 2 (the TTQRT weight).  Returns the list in
    (start time, row) order."""
    rows = list(range(k, p))
    zeroed = set()
    busy = {i: 0 for i in rows}
    events = sorted(set(ready[i] for i in rows))
    out = []
    pending = set(events)
    while len(zeroed) < len(rows) - 1:
        t = min(pending)
        pending.discard(t)
        avail = [i for i in rows if i not in zeroed and ready[i] <= t and busy[i] <= t]
        n = len(avail)
        if n >= 2:
            s = n // 2
            bottom = avail[n - 2 * s:]
            started = []
            for j in range(s):
                piv, i = bottom[j], bottom[s + j]
                started.append((t, i, piv))
                zeroed.add(i)
                busy[piv] = t + W_TTQRT
            pending.add(t + W_TTQRT)
            out.extend(sorted(started))
    return [(k, i, piv) for (_, i, piv) in out]


def grasap(p: int, q: int, n_asap: int = 1):
    """GrASAP(n_asap) (Definition 'grasap'): Greedy on the first q - n_asap columns,
    ASAP on the last n_asap columns, driven by the simulated finish times of GEQRT.
    GrASAP = GrASAP(1); ASAP = GrASAP(q).  For p <= q the last column has nothing to
    zero, and GrASAP is read as Greedy."""
    kmax = min(p, q)
    greedy_list, _ = greedy_coarse(p, q)
    first_asap = q - n_asap if p > q else kmax
    if n_asap >= q:
        first_asap = 0
    sched = TileSchedule()
    out = []
    for k in range(kmax):
        g = _column_panel(sched, p, q, k)
        if k < first_asap:
            col = [e for e in greedy_list if e[0] == k]
        else:
            col = asap_column(p, k, g)
        _column_elims(sched, q, k, col)
        out.extend(col)
    return out


def elimination_list(p: int, q: int, tree: int, bs: int = 1):
    """The elimination list of one of the trees, in canonical order."""
    if p < 1 or q < 1:
        raise ValueError("p and q must be >= 1")
    if tree == FLAT:
        return flat_tree(p, q)
    if tree == PLASMA:
        return plasma_tree(p, q, bs)
    if tree == BINARY:
        return binary_tree(p, q)
    if tree == FIBONACCI:
        return fibonacci_coarse(p, q)[0]
    if tree == GREEDY:
        return greedy_coarse(p, q)[0]
    if tree == GRASAP:
        return grasap(p, q, 1)
    if tree == ASAP:
        return grasap(p, q, q)
    raise ValueError(f"unknown tree {tree}")


def check_valid(p: int, q: int, elims) -> None:
    """Raise ValueError unless the list is a valid generic tiled algorithm (Section
    3.1.2): exactly one elimination per sub-diagonal tile of the first min(p,q)
    columns; both rows ready (zeroed in every earlier column) when it runs; the pivot
    still a potential annihilator (not yet zeroed in this column)."""
    kmax = min(p, q)
    done = set()
    for (k, i, piv) in elims:
        if not (0 <= k < kmax and k < i < p and k <= piv < p and piv != i):
            raise ValueError(f"bad triple {(k, i, piv)}")
        if (i, k) in done:
            raise ValueError(f"tile {(i, k)} zeroed twice")
        for kk in range(k):
            for r in (i, piv):
                if r > kk and (r, kk) not in done:
                    raise ValueError(f"row {r} not ready for {(k, i, piv)}")
        if (piv, k) in done:
            raise ValueError(f"pivot {piv} already zeroed in column {k}")
        done.add((i, k))
    for k in range(kmax):
        for i in range(k + 1, p):
            if (i, k) not in done:
                raise ValueError(f"tile {(i, k)} never zeroed")


def schedule(p: int, q: int, elims, ts: bool = False) -> TileSchedule:
    """Simulate the whole task graph of an elimination list (its TS form when ts)."""
    sched = TileSchedule()
    by_col = {}
    for e in elims:
        by_col.setdefault(e[0], []).append(e)
    tsr = ts_rows(elims) if ts else {}
    for k in range(min(p, q)):
        _column_panel(sched, p, q, k, tsr.get(k, ()))
        _column_elims(sched, q, k, by_col.get(k, []), tsr.get(k, ()))
    return sched


def critical_path(p: int, q: int, elims, ts: bool = False) -> int:
    """Weighted critical path (unit nb^3/3), the makespan with unbounded processors."""
    return schedule(p, q, elims, ts).makespan


def tiled_table(p: int, q: int, elims):
    """tiled[(i, k)] = finish time of TTQRT(i, piv, k) (Table 'Time-steps for tiled
    algorithms')."""
    sched = schedule(p, q, elims)
    return {(i, k): sched.finish[("TTQRT", i, piv, k)] for (k, i, piv) in elims}


def kernel_counts(p: int, q: int, elims, ts: bool = False):
    """Number of tasks of each kernel in the task graph of the list (its TS form when
    ts), enumerated from the column-by-column program."""
    kmax = min(p, q)
    tsr = ts_rows(elims) if ts else {}
    c = {"GEQRT": 0, "TTQRT": 0, "UNMQR": 0, "TTMQR": 0, "TSQRT": 0, "TSMQR": 0}
    for k in range(kmax):
        panel_rows = (p - k) - len(tsr.get(k, ()))
        c["GEQRT"] += panel_rows
        c["UNMQR"] += panel_rows * (q - 1 - k)
    for (k, i, _) in elims:
        if i in tsr.get(k, ()):
            c["TSQRT"] += 1
            c["TSMQR"] += q - 1 - k
        else:
            c["TTQRT"] += 1
            c["TTMQR"] += q - 1 - k
    return c
