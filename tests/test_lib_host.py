"""Host-side tests of libtqr (no GPU): the library loads and exports every symbol that
include/tqr.h declares; its elimination lists, critical paths and task counts are
bit-exact against the oracle; invalid arguments return LAPACK-style negative codes."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import elimlists as E

import paper_1303_3182_gb300 as tqr


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1303_3182_gb300 import build
    build.build()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "tqr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tqr_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    names = _declared_symbols()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", tqr.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert missing == []
    L = ctypes.CDLL(tqr.LIB_PATH)
    for n in names:
        assert getattr(L, n) is not None


ORACLE_TREES = [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP, E.ASAP]


@pytest.mark.parametrize("tree", ORACLE_TREES)
@pytest.mark.parametrize("p,q", [(1, 1), (1, 3), (2, 2), (3, 7), (8, 2), (15, 6), (17, 5),
                                 (33, 9), (40, 40), (128, 16)])
def test_elimlist_bitexact_vs_oracle(p, q, tree):
    bs = 4
    lst, cp = tqr.elimlist(p, q, tree, bs)
    ref = E.elimination_list(p, q, tree, bs=bs)
    assert [tuple(map(int, r)) for r in lst] == ref
    if p * q <= 40 * 40:
        assert cp == E.critical_path(p, q, ref)


def test_cp_values_of_workload_shapes():
    """128 x 16 tiles (32768 x 4096 at nb = 256) with the six trees, and the thesis's
    biggermat Greedy entry 396 for that shape."""
    cps = {t: tqr.elimlist(128, 16, t, 4)[1] for t in
           ["flat", "plasma", "binary", "fibonacci", "greedy", "grasap"]}
    assert cps["greedy"] == 396
    for t, v in cps.items():
        assert v == E.critical_path(128, 16, E.elimination_list(128, 16, tqr.TREES[t], bs=4)), t


@pytest.mark.parametrize("m,n,nb", [(512, 128, 64), (1000, 300, 64), (300, 1000, 64), (64, 64, 64)])
def test_plan_stats_vs_oracle(m, n, nb):
    p, q = -(-m // nb), -(-n // nb)
    for tree in ["greedy", "flat", "fibonacci", "asap"]:
        st = tqr.plan_stats(m, n, nb, tree, 1)
        ref = E.elimination_list(p, q, tqr.TREES[tree])
        counts = E.kernel_counts(p, q, ref)
        for k in ("GEQRT", "TTQRT", "UNMQR", "TTMQR"):
            assert st[k] == counts[k]
        assert st["cp"] == E.critical_path(p, q, ref)


def test_c1_shape_counts():
    """512 x 128, nb 64: p = 8, q = 2: 15 GEQRT, 13 TTQRT, 8 UNMQR, 7 TTMQR, Greedy CP 34."""
    st = tqr.plan_stats(512, 128, 64, "greedy", 1)
    assert (st["GEQRT"], st["TTQRT"], st["UNMQR"], st["TTMQR"], st["cp"]) == (15, 13, 8, 7, 34)


def test_invalid_arguments():
    L = tqr.lib()
    n = ctypes.c_int64(0)
    assert L.tqr_elimlist(0, 3, 4, 1, None, ctypes.byref(n), None) == -1
    assert L.tqr_elimlist(3, 0, 4, 1, None, ctypes.byref(n), None) == -2
    assert L.tqr_elimlist(3, 3, 9, 1, None, ctypes.byref(n), None) == -3
    assert L.tqr_elimlist(3, 3, 1, 0, None, ctypes.byref(n), None) == -4
    assert L.tqr_elimlist(3, 3, 4, 1, None, None, None) == -6
    small = (ctypes.c_int32 * 3)()
    cap = ctypes.c_int64(1)
    assert L.tqr_elimlist(5, 2, 4, 1, small, ctypes.byref(cap), None) == -6
    vp = ctypes.c_void_p
    assert L.tqr_factor(0, 4, 4, 2, 4, 1, 0, vp(8), 4, vp(8), None) == -1
    assert L.tqr_factor(8, 4, 0, 2, 4, 1, 0, vp(8), 8, vp(8), None) == -3
    assert L.tqr_factor(8, 4, 4, 5, 4, 1, 0, vp(8), 8, vp(8), None) == -4
    assert L.tqr_factor(8, 4, 4, 2, 7, 1, 0, vp(8), 8, vp(8), None) == -5
    assert L.tqr_factor(8, 4, 4, 2, 1, 0, 0, vp(8), 8, vp(8), None) == -6
    assert L.tqr_factor(8, 4, 4, 2, 4, 1, 9, vp(8), 8, vp(8), None) == -7
    assert L.tqr_factor(8, 4, 4, 2, 4, 1, 0, None, 8, vp(8), None) == -8
    assert L.tqr_factor(8, 4, 4, 2, 4, 1, 0, vp(8), 7, vp(8), None) == -9
    assert L.tqr_factor(8, 4, 4, 2, 4, 1, 0, vp(8), 8, None, None) == -10
    assert L.tqr_trsm(0, 0, vp(8), 1, vp(8), 1, 1, None) == -1
    assert L.tqr_strerror(3) == b"device dependency wait exceeded the limit"
    assert L.tqr_set_column_parts(3) == -1 and L.tqr_set_column_parts(-1) == -1
    assert L.tqr_set_column_parts(1) == 0
    w9 = (ctypes.c_int64 * 9)(265, 285, 20, 32, 320, 32, 66, 80, 0)
    assert L.tqr_set_claim_order_tc(3, None) == -1
    assert L.tqr_set_claim_order_tc(1, w9) == -2
    assert L.tqr_set_claim_order_tc(2, None) == 0


def test_workspace_and_flops():
    # two ib x nb T factors per tile (i, k), k < min(p, q)
    assert tqr.workspace_size(512, 128, 64, 16, "fp64") == 2 * 8 * 2 * 16 * 64 * 8
    assert tqr.workspace_size(512, 128, 64, 16, "fp32") == 2 * 8 * 2 * 16 * 64 * 4
    assert tqr.nominal_flops(32768, 4096) == pytest.approx(2 * 4096 ** 2 * (32768 - 4096 / 3))


@pytest.mark.parametrize("m,n,nb", [(512, 128, 64), (1000, 300, 64), (300, 1000, 64), (64, 64, 64), (2048, 640, 128)])
def test_ts_plan_counts_vs_oracle(m, n, nb):
    """TS form of each tree (tree | TQR_TS): the library's task counts and critical path
    equal the oracle's TS-form schedule (TSQRT weight 6, TSMQR 12)."""
    p, q = -(-m // nb), -(-n // nb)
    for tree in ["flat", "plasma", "binary", "fibonacci", "greedy", "grasap"]:
        st = tqr.plan_counts(m, n, nb, tree + "-ts", 3)
        ref = E.elimination_list(p, q, tqr.TREES[tree], bs=3)
        counts = E.kernel_counts(p, q, ref, ts=True)
        for k in ("GEQRT", "TTQRT", "UNMQR", "TTMQR", "TSQRT", "TSMQR"):
            assert st[k] == counts[k], (tree, k)
        assert st["cp"] == E.critical_path(p, q, ref, ts=True), tree
        # the TT form through the same entry point is unchanged
        tt = tqr.plan_counts(m, n, nb, tree, 3)
        assert tt["TSQRT"] == 0 and tt["TSMQR"] == 0
        assert tt["cp"] == E.critical_path(p, q, ref)
        _, cp = tqr.elimlist(p, q, tree + "-ts", 3)
        assert cp == st["cp"]


def test_ts_claim_order_topological():
    """The executor order of a TS-form graph is a topological order of the oracle's
    TS-form program (every task after the tasks it conflicts with)."""
    for tree in ["flat-ts", "plasma-ts", "greedy-ts"]:
        for mode in (0, 1):
            order = tqr.claim_order(9, 4, tree, 3, mode=mode, nproc=5)
            names = {0: "GEQRT", 1: "TTQRT", 2: "UNMQR", 3: "TTMQR", 6: "TSQRT", 7: "TSMQR"}
            keys = []
            for kind, i, piv, k, j in order:
                nm = names[int(kind)]
                if nm == "GEQRT":
                    keys.append((nm, i, k))
                elif nm == "UNMQR":
                    keys.append((nm, i, k, j))
                elif nm in ("TTQRT", "TSQRT"):
                    keys.append((nm, i, piv, k))
                else:
                    keys.append((nm, i, piv, k, j))
            base = tqr.TREES[tree] & ~tqr.TS
            sched = E.schedule(9, 4, E.elimination_list(9, 4, base, bs=3), ts=True)
            assert sorted(keys) == sorted(sched.finish.keys())
            pos = {key: r for r, key in enumerate(keys)}
            # a task starts no earlier than its earliest-start predecessors finish: in a
            # topological order, tasks with a finish time <= another's start come first
            for key in keys:
                st = sched.finish[key] - {"GEQRT": 4, "TTQRT": 2, "UNMQR": 6, "TTMQR": 6,
                                          "TSQRT": 6, "TSMQR": 12}[key[0]]
                for other in keys:
                    if sched.finish[other] <= st and _conflict(key, other):
                        assert pos[other] < pos[key], (tree, mode, key, other)


def _regions(key):
    nm = key[0]
    if nm == "GEQRT":
        _, i, k = key
        return set(), {(i, k, "L"), (i, k, "U")}
    if nm == "UNMQR":
        _, i, k, j = key
        return {(i, k, "L")}, {(i, j, "L"), (i, j, "U")}
    if nm == "TTQRT":
        _, i, piv, k = key
        return set(), {(piv, k, "U"), (i, k, "U")}
    if nm == "TSQRT":
        _, i, piv, k = key
        return set(), {(piv, k, "U"), (i, k, "L"), (i, k, "U")}
    _, i, piv, k, j = key
    rd = {(i, k, "U")} if nm == "TTMQR" else {(i, k, "L"), (i, k, "U")}
    return rd, {(piv, j, "L"), (piv, j, "U"), (i, j, "L"), (i, j, "U")}


def _conflict(a, b):
    ra, wa = _regions(a)
    rb, wb = _regions(b)
    return bool(wa & (rb | wb)) or bool(wb & ra)


def test_complex_precision_arguments():
    """TQR_Z64: 16-byte T entries, nb <= 128, no batched form (host checks only)."""
    L = tqr.lib()
    sz = tqr.workspace_size(256, 128, 64, 16, "z64")
    assert sz == 2 * tqr.workspace_size(256, 128, 64, 16, "fp64")
    out = ctypes.c_size_t(0)
    assert L.tqr_workspace_size(256, 128, 256, 16, tqr.Z64, ctypes.byref(out)) == -3
    assert L.tqr_factor(256, 128, 256, 16, 4, 1, tqr.Z64, ctypes.c_void_p(1), 256, ctypes.c_void_p(1), None) == -3
    m = (ctypes.c_int64 * 1)(64)
    ptrs = (ctypes.c_void_p * 1)(1)
    h = ctypes.c_void_p(0)
    assert L.tqr_batch_plan_create(1, m, m, ptrs, m, None, tqr.Z64, ptrs, ctypes.byref(h)) == -7


def test_split_pairs_match_fp32_rounding():
    """The refinement's FP32 pair split (integer instructions) against its definition:
    hi = fl32(x) and lo = fl32(x - hi) rounded to nearest even by numpy, bit for bit -
    random magnitudes over the whole range, rounding ties (even and odd), carries into
    the exponent, both signs, and the values outside the integer path's range (zero,
    subnormal, tiny, huge, inf) that take the plain conversions."""
    L = tqr.lib()
    rng = np.random.default_rng(1303318210)
    parts = [rng.standard_normal(20000),
             rng.standard_normal(20000) * np.exp2(rng.integers(-80, 130, 20000)),
             np.array([0.0, -0.0, 1.0, -1.0, 5e-324, 2.0 ** -1022, 2.0 ** -75, 2.0 ** -74, 2.0 ** -73,
                       2.0 ** 126, 2.0 ** 127 * 0.999, 1e300, -1e300, np.inf, -np.inf, 3.4e38])]
    # ties at the 29-bit boundary: keep bit even / odd, and the all-ones carry
    base = np.float64(1.0) + np.arange(64) * 2.0 ** -23
    parts.append(base + 2.0 ** -24)
    parts.append(-(base + 2.0 ** -24))
    parts.append(np.nextafter(np.float64(2.0), 0.0) * np.exp2(np.arange(-60, 60)))
    x = np.ascontiguousarray(np.concatenate(parts), dtype=np.float64)
    n = x.size
    hi = np.empty(n, dtype=np.float32)
    lo = np.empty(n, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    assert L.tqr_debug_split_pairs(n, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), hi.ctypes.data_as(fp),
                                   lo.ctypes.data_as(fp)) == 0
    with np.errstate(over="ignore", invalid="ignore"):
        ref_hi = x.astype(np.float32)
        ref_lo = (x - ref_hi.astype(np.float64)).astype(np.float32)
    fin = np.isfinite(x)
    assert np.array_equal(hi.view(np.uint32)[fin], ref_hi.view(np.uint32)[fin])
    same = ref_lo.view(np.uint32) == lo.view(np.uint32)
    both_zero = (ref_lo == 0) & (lo == 0)  # +0 / -0 of an exact split are the same value
    assert np.all((same | both_zero)[fin])
    assert L.tqr_debug_split_pairs(-1, None, None, None) == -1
    assert L.tqr_debug_split_pairs(3, None, None, None) == -2
