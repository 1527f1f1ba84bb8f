"""Pins for the numeric side of the oracle (FP64 Householder and the tiled algorithm).

The thesis prints no factor values, so the oracle is pinned to the mathematics:
brute force against unblocked Householder QR and LAPACK (numpy.linalg.qr), the
definition of a QR factorization (A = QR, Q^T Q = I), the compact-WY identity
I - V T V^T = H_1 ... H_b with each reflector formed explicitly, closed forms, and
least-squares optimality.
"""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H
from oracle import refine

ALL_TREES = [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP, E.ASAP]


def _explicit_reflector(v, tau):
    return np.eye(len(v)) - tau * np.outer(v, v)


def test_householder_reflector():
    rng = np.random.default_rng(1)
    for alpha in (1.5, -0.7, 0.0):
        x = rng.standard_normal(6)
        beta, tau, v = H.householder(alpha, x)
        vv = np.concatenate(([1.0], v))
        Hm = _explicit_reflector(vv, tau)
        out = Hm @ np.concatenate(([alpha], x))
        assert abs(out[0] - beta) < 1e-14 * 4
        assert np.max(np.abs(out[1:])) < 1e-14 * 4
        assert np.max(np.abs(Hm @ Hm.T - np.eye(7))) < 1e-14 * 4
        assert 1.0 <= tau <= 2.0
        assert (beta < 0) == (alpha >= 0)
    beta, tau, v = H.householder(-2.0, np.zeros(3))
    assert tau == 0.0 and beta == -2.0


def _q_explicit(F, Tg, Tt, nb, ib, elims, m):
    return H.apply_qt(F, Tg, Tt, nb, ib, elims, np.eye(m), transpose=False)


CASES = [  # (m, n, nb, ib)
    (8, 8, 2, 1), (12, 6, 3, 2), (16, 8, 4, 2), (13, 7, 4, 3), (10, 10, 4, 4),
    (6, 4, 1, 1), (9, 5, 8, 3), (20, 12, 5, 5), (7, 9, 3, 2), (4, 4, 8, 8),
]


@pytest.mark.parametrize("m,n,nb,ib", CASES)
@pytest.mark.parametrize("tree", ALL_TREES)
def test_tiled_qr_brute_force(m, n, nb, ib, tree):
    """Tiled QR with every tree vs unblocked Householder and LAPACK: |R| equal (R is
    unique up to row signs), A = QR and Q^T Q = I to FP64 rounding."""
    A = synthetic.gaussian(m, n, seed=m * 100 + n)
    p, q = H.tile_grid(m, n, nb)
    elims = E.elimination_list(p, q, tree, bs=2)
    F, Tg, Tt = H.tiled_qr(A, nb, ib, elims)
    k = min(m, n)
    R_tiled = np.triu(F[:k, :n])
    Fu, tau = H.qr_unblocked(A)
    R_unb = np.triu(Fu[:k, :n])
    R_lapack = np.linalg.qr(A, mode="r")[:k, :n]
    scale = np.linalg.norm(A)
    tol = 1e-14 * scale * max(m, n)
    assert np.max(np.abs(np.abs(R_tiled) - np.abs(R_unb))) < tol
    assert np.max(np.abs(np.abs(R_tiled) - np.abs(R_lapack))) < tol
    Q = _q_explicit(F, Tg, Tt, nb, ib, elims, m)
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) < 1e-14 * m * 4
    Rfull = np.zeros((m, n))
    Rfull[:k] = R_tiled
    assert np.linalg.norm(A - Q @ Rfull) / scale < 1e-14 * max(m, n)
    # Q^T A reproduces R exactly in structure (zeros below the diagonal)
    QtA = H.apply_qt(F, Tg, Tt, nb, ib, elims, A)
    assert np.max(np.abs(QtA - Rfull)) < tol


def test_unblocked_qr_definition():
    A = synthetic.gaussian(9, 5, seed=3)
    F, tau = H.qr_unblocked(A)
    Q = H.form_q(F, tau)
    R = np.triu(F)
    assert np.max(np.abs(Q @ R - A)) < 1e-14 * 20
    assert np.max(np.abs(Q.T @ Q - np.eye(9))) < 1e-14 * 20


@pytest.mark.parametrize("nb,ib", [(6, 2), (6, 4), (5, 5), (7, 3)])
def test_t_factor_identity(nb, ib):
    """I - V T_b V^T equals the product of the block's reflectors, each formed from its
    vector and tau: for GEQRT and for TTQRT."""
    rng = np.random.default_rng(nb * 10 + ib)
    A = rng.standard_normal((nb, nb))
    A_work = A.copy()
    T = H.geqrt(A_work, ib)
    V = np.tril(A_work, -1) + np.eye(nb)
    for b0 in range(0, nb, ib):
        b1 = min(b0 + ib, nb)
        Tb = T[:b1 - b0, b0:b1]
        prod = np.eye(nb)
        for c in range(b0, b1):
            prod = prod @ _explicit_reflector(V[:, c], T[c - b0, c])
        assert np.max(np.abs(np.eye(nb) - V[:, b0:b1] @ Tb @ V[:, b0:b1].T - prod)) < 1e-14 * nb
        assert np.allclose(np.tril(Tb, -1), 0)
    # TTQRT: the implicit reflectors are [e_c; A2[0:c+1, c]]
    R1 = np.triu(rng.standard_normal((nb, nb)))
    A2 = np.triu(rng.standard_normal((nb, nb)))
    S = np.vstack([R1, A2])
    R1w, A2w = R1.copy(), A2.copy()
    T2 = H.ttqrt(R1w, A2w, ib)
    V2 = np.vstack([np.eye(nb), np.triu(A2w)])
    full = np.eye(2 * nb)
    for b0 in range(0, nb, ib):
        b1 = min(b0 + ib, nb)
        Tb = T2[:b1 - b0, b0:b1]
        prod = np.eye(2 * nb)
        for c in range(b0, b1):
            prod = prod @ _explicit_reflector(V2[:, c], T2[c - b0, c])
        assert np.max(np.abs(np.eye(2 * nb) - V2[:, b0:b1] @ Tb @ V2[:, b0:b1].T - prod)) \
            < 1e-14 * nb * 2
        full = full @ prod
    # Q^T [R1; A2] = [R_new; 0] and |R_new| = |R of the stacked matrix|
    out = full.T @ S
    assert np.max(np.abs(out[nb:])) < 1e-13
    assert np.max(np.abs(np.abs(np.triu(R1w)) - np.abs(np.linalg.qr(S, mode="r")))) < 1e-13


def test_closed_forms():
    """Orthonormal columns give |R| = I; an upper-triangular A gives |R| = |A|."""
    rng = np.random.default_rng(5)
    Qm = synthetic.haar_orthonormal(24, 8, rng)
    elims = E.elimination_list(6, 2, E.GREEDY)
    F, _, _ = H.tiled_qr(Qm, 4, 2, elims)
    assert np.max(np.abs(np.abs(np.triu(F[:8, :8])) - np.eye(8))) < 1e-14 * 30
    U = np.triu(rng.standard_normal((12, 12))) + 3 * np.eye(12)
    elims = E.elimination_list(4, 4, E.FIBONACCI)
    F, _, _ = H.tiled_qr(U, 3, 2, elims)
    assert np.max(np.abs(np.abs(np.triu(F[:12, :12])) - np.abs(U))) < 1e-13


def test_ragged_equals_padded():
    """A matrix that is not a whole number of tiles gives the leading part of the
    zero-padded problem's factors."""
    A = synthetic.gaussian(11, 7, seed=11)
    nb, ib = 4, 2
    p, q = H.tile_grid(11, 7, nb)
    elims = E.elimination_list(p, q, E.GREEDY)
    F, Tg, _ = H.tiled_qr(A, nb, ib, elims)
    Fp, Tgp, _ = H.tiled_qr(H.pad(A, nb), nb, ib, elims)
    assert np.array_equal(F, Fp)
    assert np.array_equal(F[11:, :], np.zeros((p * nb - 11, q * nb)))


@pytest.mark.parametrize("tree", [E.GREEDY, E.FLAT, E.FIBONACCI])
def test_lstsq(tree):
    """Least squares: A^T r = 0 to rounding; equal to LAPACK's lstsq; a consistent
    square system returns its solution."""
    m, n, nb, ib = 30, 12, 4, 2
    A, X, B = synthetic.least_squares_problem(m, n, 1e3, 1e-3, 3, seed=7)
    p, q = H.tile_grid(m, n, nb)
    elims = E.elimination_list(p, q, tree)
    Xo = H.lstsq(A, B, nb, ib, elims)
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    # both solvers are backward stable: the same optimality level, to a small factor
    assert refine.ls_optimality(A, Xo, B) < 10 * refine.ls_optimality(A, Xl, B) + 1e-16
    assert refine.rel_error(Xo, Xl) < 1e-12
    As = synthetic.gaussian(12, 12, seed=9)
    xs = np.arange(12.0).reshape(12, 1)
    elims = E.elimination_list(3, 3, tree)
    assert refine.rel_error(H.lstsq(As, As @ xs, 4, 2, elims), xs) < 1e-12


def test_apply_q_roundtrip():
    A = synthetic.gaussian(14, 6, seed=2)
    nb, ib = 3, 2
    p, q = H.tile_grid(14, 6, nb)
    elims = E.elimination_list(p, q, E.BINARY)
    F, Tg, Tt = H.tiled_qr(A, nb, ib, elims)
    Bm = synthetic.gaussian(14, 3, seed=4)
    back = H.apply_qt(F, Tg, Tt, nb, ib, elims,
                      H.apply_qt(F, Tg, Tt, nb, ib, elims, Bm), transpose=False)
    assert np.max(np.abs(back - Bm)) < 1e-14 * 20


def test_t_layout_diagonal_holds_tau():
    """tau of reflector c sits at T[c % ib, c] (block c // ib, LAPACK GEQRT layout)."""
    A = synthetic.gaussian(8, 8, seed=8)
    F, tau = H.qr_unblocked(A)
    Aw = np.array(A)
    T = H.geqrt(Aw, 3)
    assert np.allclose([T[c % 3, c] for c in range(8)], tau, atol=1e-14)


# ---------------------------------------------------------------------------
# TS kernels (triangle on top of square): Algorithm 'elimSQ', Table 'Kernels for tiled QR'
# ---------------------------------------------------------------------------

TS_TREES = [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP]


@pytest.mark.parametrize("m,n,nb,ib", CASES)
@pytest.mark.parametrize("tree", TS_TREES)
def test_ts_form_brute_force(m, n, nb, ib, tree):
    """The TS form of every list vs unblocked Householder and LAPACK: |R| equal, A = QR
    and Q^T Q = I to FP64 rounding, Q^T A = R."""
    A = synthetic.gaussian(m, n, seed=m * 100 + n + 7)
    p, q = H.tile_grid(m, n, nb)
    elims = E.elimination_list(p, q, tree, bs=2)
    F, Tg, Tt = H.tiled_qr(A, nb, ib, elims, ts=True)
    k = min(m, n)
    R_ts = np.triu(F[:k, :n])
    R_lapack = np.linalg.qr(A, mode="r")[:k, :n]
    Fu, _ = H.qr_unblocked(A)
    scale = np.linalg.norm(A)
    tol = 1e-14 * scale * max(m, n)
    assert np.max(np.abs(np.abs(R_ts) - np.abs(R_lapack))) < tol
    assert np.max(np.abs(np.abs(R_ts) - np.abs(np.triu(Fu[:k, :n])))) < tol
    Q = H.apply_qt(F, Tg, Tt, nb, ib, elims, np.eye(m), transpose=False, ts=True)
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) < 1e-14 * m * 4
    Rfull = np.zeros((m, n))
    Rfull[:k] = R_ts
    assert np.linalg.norm(A - Q @ Rfull) / scale < 1e-14 * max(m, n)
    QtA = H.apply_qt(F, Tg, Tt, nb, ib, elims, A, ts=True)
    assert np.max(np.abs(QtA - Rfull)) < tol


@pytest.mark.parametrize("nb,ib,mb", [(6, 2, 6), (6, 4, 6), (5, 5, 5), (7, 3, 7), (6, 4, 3)])
def test_tsqrt_t_identity_and_definition(nb, ib, mb):
    """TSQRT's T: I - V T_b V^T equals the product of its block's reflectors, each formed
    explicitly from [e_c; A2[:, c]] and tau; the reflectors map [R1; A2] to [R; 0] with
    |R| the R of the stacked matrix (mb < nb: a ragged bottom tile)."""
    rng = np.random.default_rng(nb * 100 + ib * 10 + mb)
    R1 = np.triu(rng.standard_normal((nb, nb)))
    A2 = rng.standard_normal((mb, nb))
    S = np.vstack([R1, A2])
    R1w, A2w = R1.copy(), A2.copy()
    T = H.tsqrt(R1w, A2w, ib)
    V = np.vstack([np.eye(nb), A2w])
    full = np.eye(nb + mb)
    for b0 in range(0, nb, ib):
        b1 = min(b0 + ib, nb)
        Tb = T[:b1 - b0, b0:b1]
        assert np.allclose(np.tril(Tb, -1), 0)
        prod = np.eye(nb + mb)
        for c in range(b0, b1):
            prod = prod @ _explicit_reflector(V[:, c], T[c - b0, c])
        assert np.max(np.abs(np.eye(nb + mb) - V[:, b0:b1] @ Tb @ V[:, b0:b1].T - prod)) < 1e-14 * nb * 4
        full = full @ prod
    out = full.T @ S
    assert np.max(np.abs(out[nb:])) < 1e-13
    assert np.max(np.abs(out[:nb] - np.triu(R1w))) < 1e-13
    assert np.max(np.abs(np.abs(np.triu(R1w)) - np.abs(np.linalg.qr(S, mode="r")))) < 1e-13
    # TSMQR applies the same transformation to any pair of blocks
    C1 = rng.standard_normal((nb, 3))
    C2 = rng.standard_normal((mb, 3))
    want = full.T @ np.vstack([C1, C2])
    H.tsmqr(A2w, T, C1, C2, ib)
    assert np.max(np.abs(np.vstack([C1, C2]) - want)) < 1e-13


def test_ts_splits_into_two_tt_kernels():
    """A TS elimination can be replaced by GEQRT of the square tile followed by TTQRT
    (Section 3.1.1): the TS form and the TT form of one list give the same |R|."""
    for tree in TS_TREES:
        for (m, n, nb) in [(40, 24, 8), (33, 17, 6)]:
            A = synthetic.gaussian(m, n, seed=tree + m)
            p, q = H.tile_grid(m, n, nb)
            elims = E.elimination_list(p, q, tree, bs=2)
            F_ts, _, _ = H.tiled_qr(A, nb, 3, elims, ts=True)
            F_tt, _, _ = H.tiled_qr(A, nb, 3, elims)
            k = min(m, n)
            d = np.abs(np.abs(np.triu(F_ts[:k, :n])) - np.abs(np.triu(F_tt[:k, :n])))
            assert np.max(d) < 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("tree", TS_TREES)
def test_ts_lstsq(tree):
    m, n = 60, 20
    A, X, B = synthetic.least_squares_problem(m, n, 1e2, 1e-3, 2, seed=55)
    p, q = H.tile_grid(m, n, 8)
    elims = E.elimination_list(p, q, tree, bs=3)
    Xo = H.lstsq(A, B, 8, 4, elims, ts=True)
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    assert refine.rel_error(Xo, Xl) < 1e-12
