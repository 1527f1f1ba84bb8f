"""Host-side tests of the batched entry points (no GPU): size-class tuning, workspace
offsets and the merged claim order of a batch.

The merged order must contain every task of every matrix once and keep each matrix's
own executor order (which is topological: earliest start grows along every edge), so
that the single ticket counter of the persistent executor cannot deadlock."""
import ctypes

import numpy as np
import pytest

import synthetic
import paper_1303_3182_gb300 as tqr


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1303_3182_gb300 import build
    build.build()


def _tasks_of(m, n, nb, tree, bs):
    st = tqr.plan_stats(m, n, nb, tree, bs)
    return st["GEQRT"] + st["TTQRT"] + st["UNMQR"] + st["TTMQR"]


def test_builtin_size_classes_and_table_override():
    ms, ns = [256, 8192, 100, 5000, 20], [32, 256, 100, 64, 64]
    p = tqr.batch_params(ms, ns, "fp32")
    assert [tuple(r) for r in p] == [(256, 32, 4, 1), (256, 32, 4, 1), (100, 32, 4, 1), (256, 32, 4, 1),
                                     (20, 20, 4, 1)]
    for prec in ("bf16x6", "bf16x3", "bf16", "fp16"):
        assert all(r[0] == 128 for r in tqr.batch_params(ms, ns, prec))
    table = [[0, 10 ** 9, 33, 64, 48, 16, 2, 1],      # n in 33..64 -> nb 48, binary
             [0, 1000, 0, 10 ** 9, 16, 8, 1, 3]]      # small m -> nb 16, plasma bs 3
    p = tqr.batch_params(ms, ns, "fp32", table=table)
    assert tuple(p[3]) == (48, 16, 2, 1) and tuple(p[4]) == (48, 16, 2, 1)  # first row wins
    assert tuple(p[0]) == (16, 8, 1, 3) and tuple(p[2]) == (16, 8, 1, 3)
    assert tuple(p[1]) == (256, 32, 4, 1)  # no row covers it: built-in rule


def test_workspace_offsets():
    ms, ns = [256, 8192, 100, 5000], [32, 256, 100, 64]
    for prec in ("fp32", "fp64", "bf16x6"):
        p = tqr.batch_params(ms, ns, prec)
        off = tqr.batch_workspace_offsets(ms, ns, prec, p)
        assert off[0] == 0 and np.all(off % 256 == 0)
        for b in range(len(ms)):
            need = tqr.workspace_size(ms[b], ns[b], int(p[b][0]), int(p[b][1]), prec)
            assert need <= off[b + 1] - off[b] < need + 256


@pytest.mark.parametrize("slots", [1, 152, 304, 100000])
def test_merged_order_keeps_every_matrix_order(slots):
    shapes = synthetic.ragged_batch_shapes(300, seed=21, m_lo=1, m_hi=3000, n_choices=(1, 32, 64, 100, 256))
    ms, ns = [m for m, _ in shapes], [n for _, n in shapes]
    rng = np.random.default_rng(2)
    params = []
    for m, n in shapes:
        nb = int(rng.choice([8, 32, 64, 128]))
        tree = int(rng.integers(0, 7))
        params.append([nb, min(nb, int(rng.choice([4, 16, 32]))), tree, int(rng.integers(1, 4))])
    params = np.asarray(params, dtype=np.int32)
    mat, loc = tqr.batch_order(ms, ns, "fp64", params, slots=slots)
    counts = [_tasks_of(m, n, int(p[0]), int(p[2]), int(p[3])) for (m, n), p in zip(shapes, params)]
    assert len(mat) == sum(counts)
    for b in range(len(shapes)):
        own = loc[mat == b]
        assert np.array_equal(own, np.arange(counts[b])), f"matrix {b}: own order not kept"


def test_single_matrix_order_is_its_own():
    mat, loc = tqr.batch_order([1000], [300], "fp64", [[64, 16, 4, 1]], slots=152)
    assert np.all(mat == 0) and np.array_equal(loc, np.arange(len(loc)))


def test_longest_critical_path_starts_first():
    # one tall wide matrix among small ones: its first task is claimed first
    ms, ns = [300, 300, 8192, 300], [32, 32, 256, 32]
    mat, _ = tqr.batch_order(ms, ns, "fp32", None, slots=152)
    assert mat[0] == 2


def test_batched_invalid_arguments():
    L = tqr.lib()
    i64 = ctypes.c_int64
    one = (i64 * 1)(64)
    out = (ctypes.c_int * 4)()
    assert L.tqr_batch_params(0, one, one, 4, None, 0, out) == -1
    assert L.tqr_batch_params(1, one, one, 9, None, 0, out) == -7
    bad = (i64 * 8)(0, 100, 0, 100, 64, 48, 4, 1)  # ib > 32
    assert L.tqr_batch_params(1, one, one, 4, bad, 1, out) == -3
    zero = (i64 * 1)(0)
    assert L.tqr_batch_params(1, zero, one, 4, None, 0, out) == -2
    cnt = i64(0)
    assert L.tqr_batch_order(1, one, one, 4, None, 152, None, None, None) == -4
    assert L.tqr_batch_order(1, one, one, 4, None, 152, None, None, ctypes.byref(cnt)) == 0
    assert cnt.value == 1  # a 64 x 64 matrix at nb 64: one GEQRT
    plan = ctypes.c_void_p(0)
    assert L.tqr_batch_plan_create(0, one, one, None, one, None, 4, None, ctypes.byref(plan)) == -1
