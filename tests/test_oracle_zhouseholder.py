"""Pins for the double-complex oracle (the thesis's second precision, Section 3.3).

As for the real oracle, the thesis prints no factor values; the complex oracle is pinned
to the mathematics and to LAPACK: the reflector's defining property H^H [alpha; x] =
[beta; 0] with real beta and unitary H; brute force against unblocked Householder QR and
numpy's (LAPACK's) complex QR (|R| equal: R is unique up to a unit-modulus factor per
row); A = QR, Q^H Q = I; the compact-WY identity I - V T V^H = H_1 ... H_b; least squares
against numpy; and on real input the complex oracle reduces to the real one."""
import numpy as np
import pytest

import synthetic
from oracle import elimlists as E
from oracle import householder as H
from oracle import zhouseholder as Z

TREES = [E.FLAT, E.PLASMA, E.BINARY, E.FIBONACCI, E.GREEDY, E.GRASAP]


def _refl(v, tau):
    return np.eye(len(v)) - tau * np.outer(v, np.conj(v))


def test_zhouseholder_definition():
    rng = np.random.default_rng(3)
    for alpha in (1.5 - 0.5j, -0.7 + 2j, 0.0 + 0j, 0.3j):
        x = rng.standard_normal(5) + 1j * rng.standard_normal(5)
        beta, tau, v = Z.zhouseholder(alpha, x)
        vv = np.concatenate(([1.0], v))
        Hm = _refl(vv, tau)
        out = Hm.conj().T @ np.concatenate(([alpha], x))
        assert abs(out[0] - beta) < 1e-14 * 8 and abs(np.imag(beta)) == 0.0
        assert np.max(np.abs(out[1:])) < 1e-14 * 8
        assert np.max(np.abs(Hm.conj().T @ Hm - np.eye(6))) < 1e-14 * 8
        assert (beta.real < 0) == (alpha.real >= 0)
    # x = 0: tau = 0 only when alpha is real; a complex alpha still gets a reflector that
    # makes the diagonal real
    beta, tau, _ = Z.zhouseholder(-2.0 + 0j, np.zeros(3, dtype=complex))
    assert tau == 0 and beta == -2.0
    beta, tau, v = Z.zhouseholder(1.0 + 1.0j, np.zeros(3, dtype=complex))
    assert tau != 0 and abs(beta.imag) == 0 and abs(abs(beta) - np.sqrt(2.0)) < 1e-15
    Hm = _refl(np.concatenate(([1.0], v)), tau)
    assert abs((Hm.conj().T @ np.array([1 + 1j, 0, 0, 0]))[0] - beta) < 1e-15


CASES = [(8, 8, 2, 1), (12, 6, 3, 2), (16, 8, 4, 2), (13, 7, 4, 3), (20, 12, 5, 5), (9, 5, 8, 3), (7, 9, 3, 2)]


@pytest.mark.parametrize("m,n,nb,ib", CASES)
@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("ts", [False, True])
def test_ztiled_qr_brute_force(m, n, nb, ib, tree, ts):
    A = synthetic.complex_gaussian(m, n, seed=m * 31 + n)
    p, q = H.tile_grid(m, n, nb)
    elims = E.elimination_list(p, q, tree, bs=2)
    F, Tg, Tt = Z.ztiled_qr(A, nb, ib, elims, ts)
    k = min(m, n)
    R = np.triu(F[:k, :n])
    assert np.max(np.abs(np.imag(np.diag(R)))) == 0.0  # real diagonal
    Fu, _ = Z.zqr_unblocked(A)
    scale = np.linalg.norm(A)
    tol = 1e-14 * scale * max(m, n)
    assert np.max(np.abs(np.abs(R) - np.abs(np.triu(Fu[:k, :n])))) < tol
    assert np.max(np.abs(np.abs(R) - np.abs(np.linalg.qr(A, mode="r")[:k, :n]))) < tol
    Q = Z.zapply_q(F, Tg, Tt, nb, ib, elims, np.eye(m, dtype=complex), adjoint=False, ts=ts)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(m))) < 1e-14 * m * 4
    Rf = np.zeros((m, n), dtype=complex)
    Rf[:k] = R
    assert np.linalg.norm(A - Q @ Rf) / scale < 1e-14 * max(m, n)
    QhA = Z.zapply_q(F, Tg, Tt, nb, ib, elims, A, ts=ts)
    assert np.max(np.abs(QhA - Rf)) < tol


@pytest.mark.parametrize("nb,ib", [(6, 2), (6, 4), (5, 5), (7, 3)])
def test_zt_factor_identity(nb, ib):
    """I - V T V^H equals the product of each block's reflectors (GEQRT, TTQRT, TSQRT)."""
    rng = np.random.default_rng(nb * 10 + ib)

    def cg(*s):
        return rng.standard_normal(s) + 1j * rng.standard_normal(s)

    A = cg(nb, nb)
    T = Z.zgeqrt(A, ib)
    V = np.tril(A, -1) + np.eye(nb)
    R1 = np.triu(cg(nb, nb))
    A2 = np.triu(cg(nb, nb))
    T2 = Z.zttqrt(R1, A2, ib)
    V2 = np.vstack([np.eye(nb), np.triu(A2)])
    R1s = np.triu(cg(nb, nb))
    A3 = cg(nb, nb)
    T3 = Z.ztsqrt(R1s, A3, ib)
    V3 = np.vstack([np.eye(nb), A3])
    for VV, TT in ((V, T), (V2, T2), (V3, T3)):
        r = VV.shape[0]
        for b0 in range(0, nb, ib):
            b1 = min(b0 + ib, nb)
            Tb = TT[:b1 - b0, b0:b1]
            prod = np.eye(r, dtype=complex)
            for c in range(b0, b1):
                prod = prod @ _refl(VV[:, c], TT[c - b0, c])
            assert np.max(np.abs(np.eye(r) - VV[:, b0:b1] @ Tb @ VV[:, b0:b1].conj().T - prod)) < 1e-13
            assert np.allclose(np.tril(Tb, -1), 0)


def test_real_input_reduces_to_the_real_oracle():
    """On a real matrix every complex operation stays real: the complex oracle's factors
    equal the real oracle's (TT and TS forms)."""
    A = synthetic.gaussian(40, 24, seed=9)
    for ts in (False, True):
        elims = E.elimination_list(5, 3, E.GREEDY)
        Fz, Tgz, Ttz = Z.ztiled_qr(A.astype(complex), 8, 3, elims, ts)
        Fr, Tgr, Ttr = H.tiled_qr(A, 8, 3, elims, ts)
        assert np.max(np.abs(Fz - Fr)) < 1e-13
        assert np.max(np.abs(np.imag(Fz))) == 0.0
        for i in range(5):
            for k in range(3):
                for a, b in ((Tgz[i][k], Tgr[i][k]), (Ttz[i][k], Ttr[i][k])):
                    assert (a is None) == (b is None)
                    if a is not None:
                        assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("ts", [False, True])
def test_zlstsq(ts):
    rng = np.random.default_rng(12)
    A = synthetic.complex_gaussian(70, 24, seed=12)
    B = rng.standard_normal((70, 2)) + 1j * rng.standard_normal((70, 2))
    p, q = H.tile_grid(70, 24, 8)
    X = Z.zlstsq(A, B, 8, 4, E.elimination_list(p, q, E.PLASMA, bs=3), ts)
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    assert np.linalg.norm(X - Xl) / np.linalg.norm(Xl) < 1e-12
