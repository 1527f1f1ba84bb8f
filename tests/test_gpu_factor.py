"""GPU parity tests of the FP64 / FP32 tiled QR against the CPU oracle, through the C ABI.

Element-wise tolerance (FP64): every stored entry (R, the GEQRT and TTQRT reflectors, the
T factors) is a sum of at most ~2(m+n) rounded products of O(1) reflector entries and
entries of A, so GPU and oracle (different summation order) agree to
|delta| <= c * max(m, n) * u * scale with u = 2^-53; c = 64 covers the accumulation
of both sides.  scale is the largest magnitude in the compared block.
FP32 storage (norms and tau still in FP64): the same bound with u = 2^-24, c = 64.
"""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H
from oracle import refine

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


def to_dev(a, dtype=torch.float64):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).to(dtype)
    return t.cuda().t()  # column-major view, stride (1, m)


def to_np(t):
    return t.double().cpu().numpy()


def gpu_t_blocks(Tbuf, P, K, ib, nb, dtype):
    arr = Tbuf.view(dtype).cpu().double().numpy()
    return arr.reshape(K, P, 2, nb, ib)  # [k][i][which] -> (nb cols, ib rows) row-major view


def tree_and_ts(tree):
    """(oracle tree id, TS form?) of a tree name or id (TS forms carry tqr.TS)."""
    t = tqr.TREES[tree] if isinstance(tree, str) else tree
    return t & ~tqr.TS, bool(t & tqr.TS)


def compare_factor(A, nb, ib, tree, prec="fp64", bs=2):
    m, n = A.shape
    p, q = H.tile_grid(m, n, nb)
    base, ts = tree_and_ts(tree)
    elims = E.elimination_list(p, q, base, bs=bs)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    if prec != "fp64":
        A = A.astype(np.float32).astype(np.float64)  # the oracle runs on the rounded input
    F, Tg, Tt = H.tiled_qr(A, nb, ib, elims, ts)
    Ad = to_dev(A, dtype)
    T = tqr.factor(Ad, nb, ib, tree, bs, prec)
    torch.cuda.synchronize()
    G = to_np(Ad)
    u = U64 if prec == "fp64" else U32
    scale = max(1.0, np.max(np.abs(F[:m, :n])))
    tol = 64 * max(m, n) * u * scale
    err = np.max(np.abs(G - F[:m, :n]))
    assert err <= tol, f"factor mismatch {err} > {tol}"
    K = min(p, q)
    Tb = gpu_t_blocks(T, p, K, ib, nb, dtype)
    worst = 0.0
    for k in range(K):
        for i in range(k, p):
            for which, ref in ((0, Tg[i][k]), (1, Tt[i][k])):
                if ref is None:
                    continue
                got = Tb[k, i, which].T  # ib x nb
                worst = max(worst, np.max(np.abs(got - ref)))
    assert worst <= 64 * max(m, n) * u * 4, f"T mismatch {worst}"
    return Ad, T, F, elims


CASES = [
    # (m, n, nb, ib, tree)
    (512, 128, 64, 16, "greedy"),       # the 512 x 128 workload (p = 8, q = 2)
    (1000, 300, 64, 16, "greedy"),      # ragged rows and columns
    (640, 320, 64, 32, "flat"),
    (640, 320, 64, 32, "plasma"),
    (640, 320, 64, 32, "binary"),
    (640, 320, 64, 32, "fibonacci"),
    (640, 320, 64, 32, "grasap"),
    (640, 320, 64, 32, "asap"),
    (37, 21, 8, 3, "greedy"),           # tiny tiles, nb not a multiple of ib
    (200, 140, 48, 20, "fibonacci"),
    (128, 300, 64, 16, "greedy"),       # wide (p < q)
    (64, 64, 64, 32, "greedy"),         # one tile
    (2048, 64, 64, 32, "greedy"),       # one tile column (TSQR-like)
    (1024, 512, 256, 32, "greedy"),     # the 256 x 256 tile size of the large workloads
    (9, 5, 1, 1, "greedy"),             # scalar tiles
]


TS_CASES = [
    # the TS forms (TSQRT/TSMQR for the rows that never pivot), Algorithm "elimSQ"
    (512, 128, 64, 16, "flat-ts"),      # Sameh-Kuck with TS kernels
    (640, 320, 64, 32, "plasma-ts"),    # the PLASMA algorithm (bs = 2)
    (640, 320, 64, 32, "binary-ts"),
    (1000, 300, 64, 16, "greedy-ts"),   # ragged rows and columns
    (640, 320, 64, 32, "fibonacci-ts"),
    (640, 320, 64, 32, "grasap-ts"),
    (37, 21, 8, 3, "greedy-ts"),
    (128, 300, 64, 16, "flat-ts"),      # wide (p < q)
    (2048, 64, 64, 32, "flat-ts"),      # one tile column
    (1024, 512, 256, 32, "greedy-ts"),  # 256 x 256 tiles
    (1000, 520, 256, 32, "plasma-ts"),  # ragged 256 tiles (bottom tile of 232 rows)
    (9, 5, 1, 1, "flat-ts"),            # scalar tiles
]


@pytest.mark.parametrize("m,n,nb,ib,tree", CASES + TS_CASES)
def test_factor_fp64_parity(m, n, nb, ib, tree):
    A = synthetic.gaussian(m, n, seed=1303318201 + m + n)
    compare_factor(A, nb, ib, tree)


@pytest.mark.parametrize("m,n,nb,ib,tree", [(512, 128, 64, 16, "greedy"), (1000, 300, 64, 16, "asap"),
                                            (300, 200, 32, 8, "flat"), (1000, 300, 64, 16, "plasma-ts"),
                                            (300, 200, 32, 8, "flat-ts")])
def test_factor_fp32_parity(m, n, nb, ib, tree):
    A = synthetic.gaussian(m, n, seed=77 + m)
    compare_factor(A, nb, ib, tree, prec="fp32")


def test_degenerate_inputs():
    # zero matrix: every tau = 0, R = 0 (exact on both sides)
    compare_factor(np.zeros((130, 70)), 32, 8, "greedy")
    # an exactly zero column stays zero under every update: tau = 0 for its reflector
    A = synthetic.gaussian(160, 96, seed=5)
    A[:, 10] = 0.0
    compare_factor(A, 32, 16, "binary")
    # already upper triangular
    compare_factor(np.triu(synthetic.gaussian(96, 96, seed=6)), 32, 16, "fibonacci")


def test_rank_deficient_is_a_valid_qr():
    """With a repeated column the reflector after it is built from rounding noise, so
    R, V and T are not unique there; the result must still be a QR factorization."""
    m, n, nb, ib = 160, 96, 32, 16
    A = synthetic.gaussian(m, n, seed=5)
    A[:, 41] = A[:, 40]
    Ad = to_dev(A)
    T = tqr.factor(Ad, nb, ib, "binary", 2, "fp64")
    Q = _q_times(Ad, T, np.eye(m), nb, ib, "binary", 1)
    R = np.triu(to_np(Ad))
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 1e-13
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) <= 1e-13
    assert abs(R[41, 41]) <= 1e-12 * np.linalg.norm(A)


def _q_times(Ad, T, Z, nb, ib, tree, trans, prec="fp64"):
    B = to_dev(Z)
    tqr.apply_qt(Ad, T, B, nb, ib, tree, 2, prec, trans=trans)
    torch.cuda.synchronize()
    return to_np(B)


@pytest.mark.parametrize("m,n,nb,ib,tree", [(512, 128, 64, 16, "greedy"), (1000, 300, 64, 16, "fibonacci"),
                                            (37, 21, 8, 3, "asap"), (1000, 300, 64, 16, "plasma-ts"),
                                            (37, 21, 8, 3, "flat-ts")])
def test_apply_q_parity_and_definition(m, n, nb, ib, tree):
    A = synthetic.gaussian(m, n, seed=11 + m)
    Ad, T, F, elims = compare_factor(A, nb, ib, tree)
    p, q = H.tile_grid(m, n, nb)
    ts = tree_and_ts(tree)[1]
    _, Tg, Tt = H.tiled_qr(A, nb, ib, elims, ts)
    Z = synthetic.gaussian(m, 5, seed=3)
    for trans in (0, 1):
        got = _q_times(Ad, T, Z, nb, ib, tree, trans)
        ref = H.apply_qt(F, Tg, Tt, nb, ib, elims, Z, transpose=(trans == 0), ts=ts)
        assert np.max(np.abs(got - ref)) <= 64 * m * U64 * np.max(np.abs(ref)) * 4
    # definition: Q explicit from the GPU, A = Q R and Q^T Q = I
    Q = _q_times(Ad, T, np.eye(m), nb, ib, tree, 1)
    k = min(m, n)
    R = np.zeros((m, n))
    R[:k] = np.triu(to_np(Ad)[:k])
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 1e-13
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) <= 1e-13


@pytest.mark.parametrize("m,n,nrhs,nb,ib,tree,cond", [(512, 128, 1, 64, 16, "greedy", 1e2),
                                                      (1000, 300, 3, 64, 16, "grasap", 1e4),
                                                      (300, 300, 2, 64, 32, "fibonacci", 1e3),
                                                      (700, 130, 40, 32, 16, "flat", 1e4),
                                                      (1000, 300, 3, 64, 16, "greedy-ts", 1e4)])
def test_lstsq_fp64(m, n, nrhs, nb, ib, tree, cond):
    """GPU least squares vs the oracle's.  Both are backward stable, so their solutions
    differ by at most the LS perturbation bound (Golub & Van Loan, Thm 5.3.1):
    |dx|/|x| <~ c u (kappa + kappa^2 |r| / (|A| |x|)) with |A|_2 = 1 here; c = 64."""
    A, X, B = synthetic.least_squares_problem(m, n, cond, 1e-3, nrhs, seed=m + nrhs)
    p, q = H.tile_grid(m, n, nb)
    base, ts = tree_and_ts(tree)
    elims = E.elimination_list(p, q, base, bs=2)
    Xo = H.lstsq(A, B, nb, ib, elims, ts)
    Xg = to_np(tqr.lstsq(to_dev(A), to_dev(B), nb, ib, tree, 2, "fp64"))
    r = B - A @ Xo
    bound = 64 * U64 * (cond + cond ** 2 * np.linalg.norm(r) / np.linalg.norm(Xo))
    assert refine.rel_error(Xg, Xo) <= bound
    assert refine.ls_optimality(A, Xg, B) <= 10 * refine.ls_optimality(A, Xo, B) + 1e-16


def test_trsm_against_back_substitution():
    n = 333
    R = np.triu(synthetic.gaussian(n, n, seed=2)) + 4 * np.eye(n)
    Bm = synthetic.gaussian(n, 37, seed=3)
    ref = H.back_substitute(R, Bm)
    Bd = to_dev(Bm)
    tqr.trsm(to_dev(R), Bd, n, "fp64")
    torch.cuda.synchronize()
    assert np.max(np.abs(to_np(Bd) - ref)) <= 1e-12 * np.max(np.abs(ref))
    # FP32 storage of R: the solve runs in FP64 on the rounded R
    R32 = R.astype(np.float32).astype(np.float64)
    Bd = to_dev(Bm)
    tqr.trsm(to_dev(R32, torch.float32), Bd, n, "fp32")
    torch.cuda.synchronize()
    ref32 = H.back_substitute(R32, Bm)
    assert np.max(np.abs(to_np(Bd) - ref32)) <= 1e-12 * np.max(np.abs(ref32))


def test_wait_timeout_reports_error_and_context_survives():
    """A task graph with one release left out: the waiting CTA gives up after the wait
    limit and the call returns TQR_ETIMEOUT instead of hanging; the next call works."""
    A = synthetic.gaussian(256, 128, seed=9)
    old = tqr.set_wait_limit_ns(200 * 10 ** 6)
    try:
        tqr.debug_drop_edge(5)
        with pytest.raises(tqr.TqrError) as ei:
            tqr.factor(to_dev(A), 32, 8, "greedy", 1, "fp64")
        assert ei.value.status == tqr.TQR_ETIMEOUT
    finally:
        tqr.set_wait_limit_ns(old)
    compare_factor(A, 32, 8, "greedy")


def test_wait_timeout_tensor_core_executor():
    """The same with the tensor-core executor (split-bf16 x3): the CTAs stop at their next
    claim, free their tensor memory and the call returns TQR_ETIMEOUT; a following mixed
    factorization of the same input is bitwise equal to one made before."""
    A = synthetic.gaussian(512, 384, seed=19)
    ws = tqr.workspace_size(512, 384, 128, 32, "bf16x3")
    ref = to_dev(A, torch.float32)
    tqr.factor(ref, 128, 32, "greedy", 1, "bf16x3", T=torch.zeros(ws, dtype=torch.uint8, device="cuda"))
    old = tqr.set_wait_limit_ns(200 * 10 ** 6)
    try:
        tqr.debug_drop_edge(7)
        with pytest.raises(tqr.TqrError) as ei:
            tqr.factor(to_dev(A, torch.float32), 128, 32, "greedy", 1, "bf16x3")
        assert ei.value.status == tqr.TQR_ETIMEOUT
    finally:
        tqr.set_wait_limit_ns(old)
    again = to_dev(A, torch.float32)
    tqr.factor(again, 128, 32, "greedy", 1, "bf16x3", T=torch.zeros(ws, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(ref, again)


def test_serialized_equals_parallel_bitwise():
    """Each task's arithmetic is fixed, so the result does not depend on the schedule:
    the factorization of the same input twice is bitwise identical."""
    A = synthetic.gaussian(777, 333, seed=21)
    a1 = to_dev(A)
    a2 = to_dev(A)
    ws = tqr.workspace_size(777, 333, 64, 16, "fp64")
    t1 = torch.zeros(ws, dtype=torch.uint8, device="cuda")  # unwritten slots compare equal
    t2 = torch.zeros(ws, dtype=torch.uint8, device="cuda")
    tqr.factor(a1, 64, 16, "greedy", T=t1)
    tqr.factor(a2, 64, 16, "greedy", T=t2)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(t1, t2)


@pytest.mark.parametrize("prec,nb,ib,m,n", [("fp64", 64, 16, 1000, 300), ("bf16x6", 128, 32, 1408, 640),
                                            ("fp32", 64, 16, 777, 200)])
def test_bounded_claim_order_gives_identical_factors(prec, nb, ib, m, n):
    """Claim orders of tqr_set_claim_order (unbounded earliest start, the bounded-processor
    CP-method schedule with two weight sets, the default): each task's arithmetic is
    independent of when it runs, so the factors and T are bit-identical."""
    A = synthetic.gaussian(m, n, seed=1303318207)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    out = []
    try:
        for mode, w in ((0, None), (1, (4, 2, 6, 6)), (1, (300, 320, 20, 32)), (2, None)):
            tqr.set_claim_order(mode, w)
            Ad = to_dev(A, dtype)
            T = torch.zeros(tqr.workspace_size(m, n, nb, ib, prec), dtype=torch.uint8, device="cuda")
            tqr.factor(Ad, nb, ib, "greedy", 1, prec, T=T)
            torch.cuda.synchronize()
            out.append((Ad.cpu(), T.cpu()))
    finally:
        tqr.set_claim_order(2)
    for Ad, T in out[1:]:
        assert torch.equal(Ad, out[0][0])
        assert torch.equal(T, out[0][1])


@pytest.mark.parametrize("prec,m,n,nb,ib,tree", [("fp64", 512, 128, 64, 16, "greedy"),
                                                 ("fp64", 1000, 300, 64, 16, "plasma-ts"),
                                                 ("fp64", 1000, 520, 256, 32, "plasma-ts"),
                                                 ("fp64", 200, 140, 48, 20, "fibonacci"),
                                                 ("fp32", 300, 200, 32, 8, "flat"),
                                                 ("fp32", 640, 320, 128, 32, "greedy-ts")])
def test_column_parts_bitwise_and_parity(prec, m, n, nb, ib, tree):
    """Update tasks split into column parts (tqr_set_column_parts): every column of a
    target tile gets the arithmetic of the whole-tile task, so R, the reflectors and T are
    bitwise those of the unsplit graph, and both match the oracle."""
    A = synthetic.gaussian(m, n, seed=1303318209 + m)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    out = []
    try:
        for mode in (0, 2):
            tqr.set_column_parts(mode)
            Ad = to_dev(A, dtype)
            T = torch.zeros(tqr.workspace_size(m, n, nb, ib, prec), dtype=torch.uint8, device="cuda")
            tqr.factor(Ad, nb, ib, tree, 2, prec, T=T)
            torch.cuda.synchronize()
            out.append((Ad.cpu(), T.cpu()))
        compare_factor(A, nb, ib, tree, prec=prec)
    finally:
        tqr.set_column_parts(1)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
