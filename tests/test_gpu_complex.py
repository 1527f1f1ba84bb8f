"""GPU parity of the double-complex tiled QR (TQR_Z64; the thesis's second precision,
Section 3.3) against the complex CPU oracle, through the C ABI.

Element-wise tolerance: as for FP64 (every stored entry is a sum of at most ~2(m+n)
rounded complex products of O(1) entries, each complex operation within a few u of
exact), |delta| <= c max(m, n) u scale, u = 2^-53, c = 64 (x 4 for T)."""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H
from oracle import zhouseholder as Z

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1303_3182_gb300 as tqr  # noqa: E402

U64 = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_3182_gb300 import build
    build.build()


def to_dev(a):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.complex128).T))
    return t.cuda().t()


def tree_and_ts(tree):
    t = tqr.TREES[tree]
    return t & ~tqr.TS, bool(t & tqr.TS)


CASES = [(256, 128, 64, 16, "greedy"), (300, 170, 64, 16, "fibonacci"), (256, 192, 32, 8, "plasma-ts"),
         (200, 100, 32, 32, "flat-ts"), (128, 200, 64, 16, "greedy"), (37, 21, 8, 3, "binary"),
         (512, 256, 128, 32, "greedy-ts"), (9, 5, 1, 1, "flat")]


@pytest.mark.parametrize("m,n,nb,ib,tree", CASES)
def test_complex_factor_parity(m, n, nb, ib, tree):
    A = synthetic.complex_gaussian(m, n, seed=7000 + m + n)
    p, q = H.tile_grid(m, n, nb)
    base, ts = tree_and_ts(tree)
    elims = E.elimination_list(p, q, base, bs=2)
    F, Tg, Tt = Z.ztiled_qr(A, nb, ib, elims, ts)
    Ad = to_dev(A)
    T = tqr.factor(Ad, nb, ib, tree, 2, "z64")
    torch.cuda.synchronize()
    G = Ad.cpu().numpy()
    scale = max(1.0, np.max(np.abs(F[:m, :n])))
    tol = 64 * max(m, n) * U64 * scale
    assert np.max(np.abs(G - F[:m, :n])) <= tol
    K = min(p, q)
    Tb = T.view(torch.complex128).cpu().numpy().reshape(K, p, 2, nb, ib)
    worst = 0.0
    for k in range(K):
        for i in range(k, p):
            for which, ref in ((0, Tg[i][k]), (1, Tt[i][k])):
                if ref is not None:
                    worst = max(worst, np.max(np.abs(Tb[k, i, which].T - ref)))
    assert worst <= 4 * tol


@pytest.mark.parametrize("m,n,nb,ib,tree", [(256, 128, 64, 16, "greedy"), (200, 100, 32, 32, "plasma-ts")])
def test_complex_apply_q_parity_and_definition(m, n, nb, ib, tree):
    A = synthetic.complex_gaussian(m, n, seed=7100 + m)
    p, q = H.tile_grid(m, n, nb)
    base, ts = tree_and_ts(tree)
    elims = E.elimination_list(p, q, base, bs=2)
    F, Tg, Tt = Z.ztiled_qr(A, nb, ib, elims, ts)
    Ad = to_dev(A)
    T = tqr.factor(Ad, nb, ib, tree, 2, "z64")
    Bm = synthetic.complex_gaussian(m, 3, seed=5)
    for trans in (0, 1):
        Bd = to_dev(Bm)
        tqr.apply_qt(Ad, T, Bd, nb, ib, tree, 2, "z64", trans=trans)
        torch.cuda.synchronize()
        ref = Z.zapply_q(F, Tg, Tt, nb, ib, elims, Bm, adjoint=(trans == 0), ts=ts)
        assert np.max(np.abs(Bd.cpu().numpy() - ref)) <= 64 * m * U64 * np.max(np.abs(ref)) * 4
    # explicit Q from the GPU: unitary and A = Q R (R with a real diagonal)
    Qd = to_dev(np.eye(m, dtype=complex))
    tqr.apply_qt(Ad, T, Qd, nb, ib, tree, 2, "z64", trans=1)
    Q = Qd.cpu().numpy()
    R = np.zeros((m, n), dtype=complex)
    R[:n] = np.triu(Ad.cpu().numpy()[:n])
    assert np.max(np.abs(np.imag(np.diag(R)))) == 0.0
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(m))) <= 1e-13
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 1e-13


@pytest.mark.parametrize("m,n,nrhs,tree", [(300, 120, 2, "greedy"), (256, 256, 1, "plasma-ts")])
def test_complex_lstsq(m, n, nrhs, tree):
    A = synthetic.complex_gaussian(m, n, seed=7200 + m)
    B = synthetic.complex_gaussian(m, nrhs, seed=7300 + m)
    p, q = H.tile_grid(m, n, 64)
    base, ts = tree_and_ts(tree)
    Xo = Z.zlstsq(A, B, 64, 16, E.elimination_list(p, q, base, bs=2), ts)
    Xg = tqr.lstsq(to_dev(A), to_dev(B), 64, 16, tree, 2, "z64").cpu().numpy()
    kappa = np.linalg.cond(A)
    r = B - A @ Xo
    bound = 64 * U64 * (kappa + kappa ** 2 * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(Xo)))
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= bound
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    assert np.linalg.norm(Xg - Xl) / np.linalg.norm(Xl) <= bound


def test_complex_trsm():
    n = 200
    R = np.triu(synthetic.complex_gaussian(n, n, seed=8)) + 4 * np.eye(n)
    Bm = synthetic.complex_gaussian(n, 5, seed=9)
    ref = Z.zback_substitute(R, Bm)
    Bd = to_dev(Bm)
    tqr.trsm(to_dev(R), Bd, n, "z64")
    torch.cuda.synchronize()
    assert np.max(np.abs(Bd.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
