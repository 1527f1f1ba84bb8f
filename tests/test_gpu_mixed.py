"""GPU tests of the tensor-core (mixed-precision) tiled QR: FP32 matrix, FP64 Householder
norms and tau, UNMQR/TTMQR on tcgen05 with split-bf16 x3, bf16 or fp16 products and FP32
accumulation (nb = 128).

Tolerances.  A product of split operands (a = a_hi + a_lo + d_a, |a_lo| <= 2^-9 |a|,
|d_a| <= 2^-9 |a_lo|) computed as a_hi b_hi + a_hi b_lo + a_lo b_hi misses
a_lo b_lo + (rounding of the lo parts), at most 3 * 2^-18 |a||b|; with FP32 accumulation
the effective unit roundoff of one update is u_x3 ~ 2^-16.  A single bf16 product has
u = 2^-8, fp16 u = 2^-11.  Split-bf16 x6 (three parts, six products) drops only the
products of part orders >= 3 (at most 3 * 2^-24 * 2^-3 |a||b|), so its error is that of
the FP32 accumulation in tensor memory; it is taken as two FP32 units, u_x6 = 2^-23.  The
backward error of the whole factorization grows like u * sqrt(n) (normwise, random
data), so the checks use c * u * sqrt(n) with c = 8.  The FP32 parts (panels, storage)
add 2^-24-level errors that are covered by the same bounds.
"""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1303_3182_gb300 as tqr  # noqa: E402

U = {"bf16x6": 2.0 ** -23, "bf16x3": 2.0 ** -16, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "fp32": 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_3182_gb300 import build
    build.build()


def to_dev(a, dtype=torch.float64):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dtype)
    return t.cuda().t()


def to_np(t):
    return t.double().cpu().numpy()


def factor_mixed(A, prec, tree="greedy", ib=32):
    Ad = to_dev(A, torch.float32)
    m, n = A.shape
    # zero-filled so that slots no task writes (tiles above the diagonal) compare equal
    T = torch.zeros(tqr.workspace_size(m, n, 128, ib, prec), dtype=torch.uint8, device="cuda")
    tqr.factor(Ad, 128, ib, tree, 2, prec, T=T)
    torch.cuda.synchronize()
    return Ad, T


def q_explicit(Ad, T, m, tree, prec, ib=32):
    Z = to_dev(np.eye(m))
    tqr.apply_qt(Ad, T, Z, 128, ib, tree, 2, prec, trans=1)
    torch.cuda.synchronize()
    return to_np(Z)


CASES = [(640, 384, "greedy"), (700, 300, "fibonacci"), (512, 512, "flat"), (1024, 256, "asap"),
         (300, 700, "greedy"),
         # TS forms (TSQRT / TSMQR): the TSMQR operand V2 is a dense tile
         (640, 384, "greedy-ts"), (700, 300, "plasma-ts"), (512, 512, "flat-ts")]


def tree_and_ts(tree):
    t = tqr.TREES[tree]
    return t & ~tqr.TS, bool(t & tqr.TS)


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16", "fp16"])
@pytest.mark.parametrize("m,n,tree", CASES)
def test_mixed_factor_is_a_qr(m, n, tree, prec):
    """R of the tensor-core factorization against the FP64 oracle (|R| up to row signs),
    and the backward error ||A - Q R|| / ||A|| of the computed factors."""
    A = synthetic.gaussian(m, n, seed=m * 7 + n).astype(np.float32).astype(np.float64)
    Ad, T = factor_mixed(A, prec, tree)
    p, q = H.tile_grid(m, n, 128)
    base, ts = tree_and_ts(tree)
    F, _, _ = H.tiled_qr(A, 128, 32, E.elimination_list(p, q, base, bs=2), ts)
    k = min(m, n)
    R = np.triu(to_np(Ad)[:k])
    Ro = np.triu(F[:k, :n])
    tol = 8 * U[prec] * np.sqrt(n)
    rel_r = np.max(np.abs(np.abs(R) - np.abs(Ro))) / np.max(np.abs(Ro))
    assert rel_r <= tol, (rel_r, tol)
    Q = q_explicit(Ad, T, m, tree, prec)
    Rf = np.zeros((m, n))
    Rf[:k] = R
    back = np.linalg.norm(A - Q @ Rf) / np.linalg.norm(A)
    assert back <= tol, (back, tol)
    # the stored reflectors are FP32: Q is orthogonal to FP32 rounding
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) <= 64 * m * U["fp32"]


def test_mixed_t_matches_its_reflectors():
    """The stored ib-blocked T of every GEQRT equals the compact-WY T built (in FP64, by
    the oracle's recurrence) from the stored reflectors and tau = T's diagonal."""
    m, n, ib = 512, 384, 32
    A = synthetic.gaussian(m, n, seed=3).astype(np.float32).astype(np.float64)
    Ad, T = factor_mixed(A, "bf16x3", "greedy", ib)
    p, q = 4, 3
    Fg = to_np(Ad)
    tbytes = 2 * p * 3 * ib * 128 * 4
    Tg = T[:tbytes].view(torch.float32).cpu().double().numpy().reshape(3, p, 2, 128, ib)
    worst = 0.0
    for k in range(3):
        for i in range(k, p):
            Tt = Tg[k, i, 0].T
            tile = Fg[i * 128:(i + 1) * 128, k * 128:(k + 1) * 128]
            V = np.tril(tile, -1) + np.eye(128)
            tau = np.array([Tt[c % ib, c] for c in range(128)])
            ref = H.build_t(V, tau, ib)
            worst = max(worst, np.max(np.abs(ref - Tt)))
    assert worst <= 1e-4


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
def test_mixed_bitwise_repeatable(prec):
    """Every task's arithmetic is fixed, so two runs give bitwise identical factors."""
    A = synthetic.gaussian(900, 500, seed=4)
    a1, t1 = factor_mixed(A, prec)
    a2, t2 = factor_mixed(A, prec)
    assert torch.equal(a1, a2) and torch.equal(t1, t2)


def test_mixed_bf16x3_much_closer_than_bf16():
    A = synthetic.gaussian(768, 384, seed=8).astype(np.float32).astype(np.float64)
    errs = {}
    for prec in ("bf16x3", "bf16"):
        Ad, T = factor_mixed(A, prec)
        Q = q_explicit(Ad, T, 768, "greedy", prec)
        Rf = np.zeros((768, 384))
        Rf[:384] = np.triu(to_np(Ad)[:384])
        errs[prec] = np.linalg.norm(A - Q @ Rf) / np.linalg.norm(A)
    assert errs["bf16x3"] * 64 < errs["bf16"], errs


def test_mixed_bf16x6_close_to_fp32():
    """Three-part split with six products against split x3 and FP32 SIMT updates.  Each
    precision's backward error is within its derived bound c u sqrt(n) (c = 8; u_x6 =
    2^-23, u_x3 = 2^-16, FP32 updates 2^-24), and since u_x6 < u_x3 the x6 factorization
    is the more accurate one.  (No measured ratio is asserted: the bounds are worst
    cases, random data stays well below them.)"""
    A = synthetic.gaussian(768, 384, seed=12).astype(np.float32).astype(np.float64)
    errs = {}
    for prec in ("bf16x6", "bf16x3", "fp32"):
        Ad = to_dev(A, torch.float32)
        T = tqr.factor(Ad, 128, 32, "greedy", 1, prec)
        torch.cuda.synchronize()
        Q = q_explicit(Ad, T, 768, "greedy", prec)
        Rf = np.zeros((768, 384))
        Rf[:384] = np.triu(to_np(Ad)[:384])
        errs[prec] = np.linalg.norm(A - Q @ Rf) / np.linalg.norm(A)
    for prec, u in (("bf16x6", U["bf16x6"]), ("bf16x3", U["bf16x3"]), ("fp32", U["fp32"])):
        assert errs[prec] <= 8 * u * np.sqrt(384), (prec, errs)
    assert errs["bf16x6"] < errs["bf16x3"], errs


@pytest.mark.parametrize("tree", ["greedy", "plasma-ts", "flat-ts"])
@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3"])
def test_mixed_first_column_reflectors_elementwise(tree, prec):
    """Element-wise parity of the stored reflectors and T factors of tile column 0 with the
    FP64 oracle's.  No tensor-core product reaches tile column 0 (the updates only write
    columns j > k), so its GEQRT / TTQRT / TSQRT run on the rounded FP32 input with FP32
    storage and FP64-accurate norms - the FP32 SIMT bound |delta| <= 64 max(m, n) 2^-24
    scale applies (one more factor 4 for T, as in the FP32 parity tests)."""
    m, n, ib = 896, 384, 32
    A = synthetic.gaussian(m, n, seed=31).astype(np.float32).astype(np.float64)
    Ad, T = factor_mixed(A, prec, tree, ib)
    p, q = H.tile_grid(m, n, 128)
    base, ts = tree_and_ts(tree)
    F, Tg, Tt = H.tiled_qr(A, 128, ib, E.elimination_list(p, q, base, bs=2), ts)
    G = to_np(Ad)
    tol = 64 * max(m, n) * U["fp32"]
    col = slice(0, 128)
    scale = max(1.0, np.max(np.abs(F[:m, col])))
    # below the first diagonal tile every entry of tile column 0 is a reflector entry; the
    # diagonal tile's R is still to be combined by the TT eliminations, so compare all rows
    assert np.max(np.abs(G[:, col] - F[:m, col])) <= tol * scale
    K = min(p, q)
    tb = T[:2 * p * K * ib * 128 * 4].view(torch.float32).cpu().double().numpy().reshape(K, p, 2, 128, ib)
    worst = 0.0
    for i in range(p):
        for which, ref in ((0, Tg[i][0]), (1, Tt[i][0])):
            if ref is not None:
                worst = max(worst, np.max(np.abs(tb[0, i, which].T - ref)))
    assert worst <= 4 * tol, worst


@pytest.mark.parametrize("tree", ["greedy", "plasma-ts"])
def test_resident_panels_equal_the_chunked_simt_panels(tree):
    """The tensor-core path factors its panels with the tile resident in shared memory; the
    FP32 SIMT path (same nb, ib) streams the trailing columns through global memory in
    chunks.  Both run the same panel, Gram, T and block-reflector arithmetic, and no
    tensor-core product reaches tile column 0, so tile column 0 and its T factors agree bit
    for bit."""
    m, n, ib = 1024, 384, 32
    A = synthetic.gaussian(m, n, seed=41).astype(np.float32).astype(np.float64)
    Ad, T = factor_mixed(A, "bf16x6", tree, ib)
    As = to_dev(A, torch.float32)
    Ts = torch.zeros(tqr.workspace_size(m, n, 128, ib, "fp32"), dtype=torch.uint8, device="cuda")
    tqr.factor(As, 128, ib, tree, 2, "fp32", T=Ts)
    torch.cuda.synchronize()
    assert torch.equal(Ad[:, :128], As[:, :128])
    p = m // 128
    nT = 2 * p * 1 * ib * 128 * 4  # the T slots of tile column 0
    assert torch.equal(T[:nT], Ts[:nT])
