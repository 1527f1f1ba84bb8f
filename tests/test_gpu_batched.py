"""Batched factorization: many independent matrices, one persistent executor launch.

Every matrix of a batch runs the task graph that tqr_factor runs for it, in an order
that keeps its own dependencies, and each task computes the same arithmetic in the same
order whatever else runs beside it.  So a batched result must equal the single-matrix
result bit for bit, and through it the oracle (same tolerances as the single-matrix
parity tests: 64 * max(m, n) * u * scale).  At the full batch size (2048 FP32 matrices,
rows 256..8192, columns 32..256) a sample of matrices is checked against the unique
QR factor with a positive diagonal (sign-normalised R of LAPACK's QR).
"""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1303_3182_gb300 as tqr  # noqa: E402

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_3182_gb300 import build
    build.build()
    tqr.set_wait_limit_ns(20 * 10 ** 9)


def to_dev(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dtype)
    return t.cuda().t()


def t_blocks(Tslice, P, K, ib, nb, dtype):
    arr = Tslice.view(dtype).cpu().double().numpy()[: 2 * P * K * ib * nb]
    return arr.reshape(K, P, 2, nb, ib)


# (m, n, nb, ib, tree, bs): ragged sizes, every tree, mixed tile sizes in one launch
MIXED_BATCH = [
    (1, 1, 1, 1, "greedy", 1),
    (5, 3, 2, 1, "flat", 1),
    (37, 21, 8, 3, "greedy", 1),
    (100, 100, 32, 8, "binary", 1),
    (300, 64, 64, 16, "plasma", 2),
    (640, 130, 64, 32, "fibonacci", 1),
    (1000, 33, 48, 20, "grasap", 1),
    (64, 200, 32, 16, "asap", 1),
    (257, 129, 128, 32, "greedy", 1),
    (700, 256, 256, 32, "greedy", 1),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_mixed_configs_match_oracle(prec):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    u = U64 if prec == "fp64" else U32
    mats, As = [], []
    for b, (m, n, nb, ib, tree, bs) in enumerate(MIXED_BATCH):
        A = synthetic.gaussian(m, n, seed=4000 + b)
        if prec == "fp32":
            A = A.astype(np.float32).astype(np.float64)
        mats.append(A)
        As.append(to_dev(A, dtype))
    params = [[nb, ib, tqr.TREES[tree], bs] for (_, _, nb, ib, tree, bs) in MIXED_BATCH]
    T, off, _ = tqr.factor_batched(As, prec, params=params)
    torch.cuda.synchronize()
    for b, (m, n, nb, ib, tree, bs) in enumerate(MIXED_BATCH):
        p, q = H.tile_grid(m, n, nb)
        elims = E.elimination_list(p, q, tqr.TREES[tree], bs=bs)
        F, Tg, Tt = H.tiled_qr(mats[b], nb, ib, elims)
        G = As[b].double().cpu().numpy()
        scale = max(1.0, np.max(np.abs(F[:m, :n])))
        err = np.max(np.abs(G - F[:m, :n]))
        assert err <= 64 * max(m, n) * u * scale, f"matrix {b}: factor mismatch {err}"
        K = min(p, q)
        Tb = t_blocks(T[int(off[b]):int(off[b + 1])], p, K, ib, nb, dtype)
        for k in range(K):
            for i in range(k, p):
                for which, ref in ((0, Tg[i][k]), (1, Tt[i][k])):
                    if ref is None:
                        continue
                    d = np.max(np.abs(Tb[k, i, which].T - ref))
                    assert d <= 64 * max(m, n) * u * 4, f"matrix {b}: T mismatch {d}"


@pytest.mark.parametrize("prec", ["fp32", "bf16x6", "bf16x3"])
def test_batched_bitwise_equals_single(prec):
    """Built-in size classes; every matrix (A and its whole T workspace) equals its own
    tqr_factor result bit for bit."""
    if prec == "fp32":
        shapes = synthetic.ragged_batch_shapes(24, seed=11, m_lo=1, m_hi=900,
                                               n_choices=(1, 7, 32, 64, 100, 128, 200))
    else:
        shapes = synthetic.ragged_batch_shapes(10, seed=12, m_lo=100, m_hi=900, n_choices=(7, 32, 128, 200))
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    src = [tqr.colmajor(torch.randn(m, n, dtype=torch.float32, device="cuda", generator=g)) for m, n in shapes]
    As = [tqr.colmajor(a.clone()) for a in src]
    ms, ns = [m for m, _ in shapes], [n for _, n in shapes]
    params = tqr.batch_params(ms, ns, prec)
    off = tqr.batch_workspace_offsets(ms, ns, prec, params)
    T = torch.zeros(int(off[-1]), dtype=torch.uint8, device="cuda")
    tqr.factor_batched(As, prec, params=params, T=T)
    torch.cuda.synchronize()
    for b, (m, n) in enumerate(shapes):
        nb, ib, tree, bs = (int(x) for x in params[b])
        A1 = tqr.colmajor(src[b].clone())
        T1 = torch.zeros(tqr.workspace_size(m, n, nb, ib, prec), dtype=torch.uint8, device="cuda")
        tqr.factor(A1, nb, ib, tree, bs, prec, T=T1)
        torch.cuda.synchronize()
        assert torch.equal(As[b], A1), f"matrix {b} ({m}x{n}, nb {nb}): batched != single"
        assert torch.equal(T[int(off[b]):int(off[b]) + T1.numel()], T1), f"matrix {b}: T differs"


def test_batched_plan_graph_replay_is_bitwise_repeatable():
    shapes = [(513, 64), (1000, 128), (77, 32), (4096, 256), (300, 300)]
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    src = [tqr.colmajor(torch.randn(m, n, dtype=torch.float32, device="cuda", generator=g)) for m, n in shapes]
    As = [tqr.colmajor(a.clone()) for a in src]
    plan = tqr.BatchPlan(As, "fp32")
    plan.run(use_graph=False)
    ref = [a.clone() for a in As]
    for rep in range(2):
        for a, s in zip(As, src):
            a.copy_(s)
        plan.run(use_graph=True)
        torch.cuda.synchronize()
        for b in range(len(As)):
            assert torch.equal(As[b], ref[b]), f"replay {rep}, matrix {b}"
    info = plan.info()
    assert info["graph"] and info["matrices"] == len(shapes) and info["tasks"] > 0
    plan.close()


def test_batched_rejects_bad_arguments():
    a = tqr.colmajor(torch.zeros(64, 32, dtype=torch.float32, device="cuda"))
    with pytest.raises(tqr.TqrError):
        tqr.factor_batched([a], "fp32", params=[[0, 1, 4, 1]])
    with pytest.raises(tqr.TqrError):
        tqr.factor_batched([a], "bf16x6", params=[[64, 32, 4, 1]])  # tensor path needs nb 128
    with pytest.raises(tqr.TqrError):
        tqr.batch_params([64], [32], "fp32", table=[[0, 100, 0, 100, 64, 48, 4, 1]])  # ib > 32


def _r_positive(R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return R * d[:, None]


def test_batched_full_size_sample_against_unique_r():
    """The full 2048-matrix FP32 batch (rows uniform in [256, 8192], columns in
    {32, 64, 128, 256}) as the benchmark runs it: one graph-replayed launch.  Sixteen
    sampled matrices: sign-normalised R equals LAPACK's (the unique R with positive
    diagonal).  Tolerance: the first-order perturbation bound of R,
    ||dR|| <~ kappa_2(A) ||dA||, with a normwise backward error ||dA|| of
    16 sqrt(m n) u32 ||A||_2 (a kernel mistake gives O(||A||) errors)."""
    shapes = synthetic.ragged_batch_shapes(2048, seed=synthetic.SEED_BASE + 4)
    total = sum(m * n for m, n in shapes)
    buf = torch.empty(total, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(synthetic.SEED_BASE + 4)
    buf.normal_(generator=g)
    src = buf.clone()
    As, o = [], 0
    for m, n in shapes:
        As.append(buf[o:o + m * n].view(n, m).t())
        o += m * n
    plan = tqr.BatchPlan(As, "fp32")
    plan.run(use_graph=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    pick = sorted(set(rng.choice(len(shapes), size=16, replace=False).tolist()) | {0, len(shapes) - 1})
    o_of = np.cumsum([0] + [m * n for m, n in shapes])
    for b in pick:
        m, n = shapes[b]
        A0 = src[o_of[b]:o_of[b] + m * n].view(n, m).t().double().cpu().numpy()
        Rg = np.triu(As[b].double().cpu().numpy()[:n, :n])
        Rl = np.linalg.qr(A0, mode="r")
        s = np.linalg.svd(A0, compute_uv=False)
        tol = 16 * np.sqrt(m * n) * U32 * s[0] * (s[0] / s[-1])
        err = np.max(np.abs(_r_positive(Rg) - _r_positive(Rl)))
        assert err <= tol, f"matrix {b} ({m}x{n}): {err} > {tol}"
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_factor_batched_null_params_autotunes(prec):
    """tqr_factor_batched with params NULL (through the C ABI): the library tunes each size
    class of the batch by device timing (tqr_batch_autotune: tile size, inner block, tree)
    and factors every matrix with its class's setting.  The table has one row per class
    (row bucket x column count) with settings tqr_factor accepts; every matrix's result
    equals tqr_factor's with the same setting bit for bit; a second call takes the cached
    table."""
    shapes = [(300, 32)] * 5 + [(2000, 64)] * 3 + [(5000, 128)] * 2 + [(700, 32)] * 2
    dtype = torch.float32
    mats = [synthetic.gaussian(m, n, seed=6100 + b).astype(np.float32).astype(np.float64)
            for b, (m, n) in enumerate(shapes)]
    As = [to_dev(A, dtype) for A in mats]
    T, off, params = tqr.factor_batched(As, prec)  # params None -> NULL -> autotuned
    torch.cuda.synchronize()
    ms, ns = [m for m, _ in shapes], [n for _, n in shapes]
    table = tqr.batch_autotune(ms, ns, prec)
    assert np.array_equal(table, tqr.batch_autotune(ms, ns, prec))  # cached
    classes = {(0 if m <= 1024 else (1 if m <= 4096 else 2), n) for m, n in shapes}
    assert len(table) == len(classes)
    for row in table:
        nb, ib, tree, bs = (int(x) for x in row[4:])
        assert ib <= nb and ib <= 32 and (nb == 128 if prec != "fp32" else nb in (32, 64, 128, 256))
    for b, (m, n) in enumerate(shapes):
        row = [r for r in table if r[0] <= m <= r[1] and r[2] <= n <= r[3]]
        assert len(row) == 1 and list(params[b]) == [int(x) for x in row[0][4:]]
        nb, ib, tree, bs = (int(x) for x in params[b])
        ref = to_dev(mats[b], dtype)
        tqr.factor(ref, nb, ib, tree, bs, prec)
        torch.cuda.synchronize()
        assert torch.equal(ref, As[b]), b


def test_batched_wait_timeout_reports_error_and_context_survives():
    """A batch plan built with one merged dependency release left out (tqr_debug_drop_edge):
    the waiting CTA gives up after the wait limit, the run returns TQR_ETIMEOUT through the
    plan's status, and a following batch of the same matrices factors as before."""
    shapes = [(300, 64), (520, 128), (256, 32)]
    mats = [synthetic.gaussian(m, n, seed=6300 + b).astype(np.float32).astype(np.float64)
            for b, (m, n) in enumerate(shapes)]
    params = [[64, 16, tqr.GREEDY, 1]] * len(shapes)
    ref = [to_dev(A, torch.float32) for A in mats]
    tqr.factor_batched(ref, "fp32", params=params)
    torch.cuda.synchronize()
    old = tqr.set_wait_limit_ns(200 * 10 ** 6)
    try:
        tqr.debug_drop_edge(3)
        with pytest.raises(tqr.TqrError) as ei:
            tqr.factor_batched([to_dev(A, torch.float32) for A in mats], "fp32", params=params)
        assert ei.value.status == tqr.TQR_ETIMEOUT
    finally:
        tqr.set_wait_limit_ns(old)
        tqr.debug_drop_edge(-1)
    again = [to_dev(A, torch.float32) for A in mats]
    tqr.factor_batched(again, "fp32", params=params)
    torch.cuda.synchronize()
    for a, b in zip(ref, again):
        assert torch.equal(a, b)
