"""Host-side tests of the library's bounded-processor schedule (no GPU): tqr_schedule's
CP-method makespan, ALAP Derived bound and lost area are bit-exact against the oracle
(oracle/schedule.py, itself pinned to the thesis's 5 x 5 schedule-length table) on the
thesis weights and on other weights; invalid arguments return negative codes."""
import random

import pytest

from oracle import elimlists as E
from oracle import schedule as S

import paper_1303_3182_gb300 as tqr

TREES = {"flat": E.FLAT, "plasma": E.PLASMA, "binary": E.BINARY, "fibonacci": E.FIBONACCI,
         "greedy": E.GREEDY, "grasap": E.GRASAP, "asap": E.ASAP}


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1303_3182_gb300 import build
    build.build()


def _oracle(p, q, tree, bs, nproc, weights):
    g = S.task_graph(p, q, E.elimination_list(p, q, TREES[tree], bs=bs), weights)
    ms, _ = S.list_schedule(g, nproc)
    bound, la = S.alap_bound(g, nproc)
    return ms, bound, la


@pytest.mark.parametrize("tree", ["grasap", "greedy", "fibonacci", "flat"])
def test_5x5_table_processors_1_to_14(tree):
    for nproc in range(1, 15):
        assert tqr.schedule(5, 5, tree, 1, nproc) == _oracle(5, 5, tree, 1, nproc, S.DEFAULT_WEIGHTS)


def test_random_shapes_trees_weights_and_processors():
    rng = random.Random(1303318206)
    for _ in range(60):
        p, q = rng.randint(1, 14), rng.randint(1, 8)
        tree = rng.choice(sorted(TREES))
        bs = rng.randint(1, 4)
        nproc = rng.choice([1, 2, 3, 5, 8, 13, 40, 200])
        weights = None if rng.random() < 0.3 else tuple(rng.randint(1, 40) for _ in range(4))
        got = tqr.schedule(p, q, tree, bs, nproc, weights)
        want = _oracle(p, q, tree, bs, nproc, weights or S.DEFAULT_WEIGHTS)
        assert got == want, (p, q, tree, bs, nproc, weights)


def test_gpu_scale_weights():
    """The claim-order weights of the tensor-core executor (task durations in us) on the
    128 x 16 tile grid of a 16384 x 2048 matrix: library and oracle agree."""
    w = (295, 323, 20, 32)
    assert tqr.schedule(128, 16, "greedy", 1, 152, w) == _oracle(128, 16, "greedy", 1, 152, w)


def test_invalid_arguments():
    L = tqr.lib()
    assert L.tqr_schedule(0, 3, 4, 1, 2, None, None, None, None) == -1
    assert L.tqr_schedule(3, 0, 4, 1, 2, None, None, None, None) == -2
    assert L.tqr_schedule(3, 3, 9, 1, 2, None, None, None, None) == -3
    assert L.tqr_schedule(3, 3, 1, 0, 2, None, None, None, None) == -4
    assert L.tqr_schedule(3, 3, 4, 1, 0, None, None, None, None) == -5
    assert L.tqr_schedule(3, 3, 4, 1, 2, tqr._weights4((4, 0, 6, 6)), None, None, None) == -6
    assert L.tqr_set_claim_order(3, None) == -1
    assert L.tqr_set_claim_order(-1, None) == -1
    assert L.tqr_set_claim_order(1, tqr._weights4((1, 2, -3, 4))) == -2
    assert L.tqr_set_claim_order(0, None) == 0
    assert L.tqr_set_claim_order(2, None) == 0


def _oracle_index(g):
    names = {S.GEQRT: "GEQRT", S.TTQRT: "TTQRT", S.UNMQR: "UNMQR", S.TTMQR: "TTMQR"}
    return {(names[g.kind[t]],) + tuple(g.key[t]): t for t in range(len(g))}


def _lib_order_as_oracle_indices(order, index):
    out = []
    for kind, i, piv, k, j in order.tolist():
        key = {0: ("GEQRT", i, k), 1: ("TTQRT", i, piv, k), 2: ("UNMQR", i, k, j), 3: ("TTMQR", i, piv, k, j)}[kind]
        out.append(index[key])
    return out


@pytest.mark.parametrize("p,q,tree,bs", [(5, 5, "greedy", 1), (9, 4, "flat", 1), (12, 5, "plasma", 3),
                                         (8, 8, "fibonacci", 1), (13, 6, "grasap", 1), (7, 3, "binary", 1)])
def test_claim_orders_equal_the_oracle_schedules(p, q, tree, bs):
    """The executor's claim order: mode 1 is the start order of the CP-method list schedule
    (start time, then larger Backflow priority, then program order), mode 0 the same for
    unbounded processors with the thesis weights; both are topological."""
    rng = random.Random(p * 100 + q)
    elims = E.elimination_list(p, q, TREES[tree], bs=bs)
    for mode, nproc, weights in [(0, 1, None), (1, 3, None), (1, 17, (30, 32, 2, 3)),
                                 (1, rng.randint(2, 40), tuple(rng.randint(1, 50) for _ in range(4)))]:
        g = S.task_graph(p, q, elims, weights or S.DEFAULT_WEIGHTS)
        order = _lib_order_as_oracle_indices(tqr.claim_order(p, q, tree, bs, mode, nproc, weights), _oracle_index(g))
        assert sorted(order) == list(range(len(g)))
        pos = {t: r for r, t in enumerate(order)}
        assert all(pos[d] < pos[t] for t in range(len(g)) for d in g.preds[t])
        prio = S.bottom_levels(g)
        _, start = S.list_schedule(g, nproc if mode == 1 else len(g))
        assert order == sorted(range(len(g)), key=lambda t: (start[t], -prio[t], t))


def test_bench_tile_task_bytes_match_the_oracle_kernel_counts():
    """bench.py's algorithmic bytes of the tensor-core factorization (tile-task traffic) from
    the library's plan counts equal the same sum over the oracle's kernel counts of the
    benchmark's tree (the TS form of PlasmaTree(32) and, for comparison, Greedy)."""
    import bench

    for tree, bs, ts in (("plasma-ts", 32, True), ("greedy", 1, False)):
        class Args:
            m, n, prec = 32768, 4096, "bf16x6"
        Args.tree, Args.bs = tree, bs
        p, q = 256, 32
        base = E.PLASMA if tree.startswith("plasma") else E.GREEDY
        c = E.kernel_counts(p, q, E.elimination_list(p, q, base, bs=bs), ts=ts)
        tile, img, tblk = 128 * 128 * 4, 3 * 128 * 128 * 2, 32 * 128 * 4
        want = (c["GEQRT"] * (2 * tile + tblk) + c["TTQRT"] * (2 * tile + tblk) + c["TSQRT"] * (3 * tile + tblk)
                + c["GEQRT"] * (tile + tblk + 2 * img) + (c["TTQRT"] + c["TSQRT"]) * (tile + tblk + 3 * img)
                + c["UNMQR"] * (2 * tile + 2 * img) + (c["TTMQR"] + c["TSMQR"]) * (4 * tile + 3 * img))
        assert bench.tile_task_bytes(Args) == want, tree


def test_split_panel_graph_schedule():
    """The tensor-core graph with operand-preparation tasks and split TT / TS panels (nine
    weights of tqr_schedule_ts): on one processor its makespan is the sum of all task
    weights (every task runs once: #GEQRT + #TTQRT + #TSQRT preparations, four blocks per
    TT / TS panel); with the blocks weighing a quarter of their panel, pipelining the blocks
    of consecutive eliminations on a pivot never lengthens the critical path."""
    p, q = 12, 4
    for tree, bs in (("plasma-ts", 4), ("greedy", 1), ("flat-ts", 1)):
        c = tqr.plan_counts(p * 128, q * 128, 128, tree, bs)
        w = [40, 20, 6, 6, 24, 6]
        prep, wtt, wts = 3, 5, 6
        one, _, _ = tqr.schedule(p, q, tree, bs, 1, w + [prep, wtt, wts])
        total = (w[0] * c["GEQRT"] + w[2] * c["UNMQR"] + w[3] * c["TTMQR"] + w[5] * c["TSMQR"]
                 + prep * (c["GEQRT"] + c["TTQRT"] + c["TSQRT"]) + 4 * wtt * c["TTQRT"] + 4 * wts * c["TSQRT"])
        assert one == total, tree
        big = 10 ** 6
        unsplit, _, _ = tqr.schedule(p, q, tree, bs, big, w + [prep])
        split, _, _ = tqr.schedule(p, q, tree, bs, big, w + [prep, w[1] // 4, w[4] // 4])
        assert split <= unsplit, tree
