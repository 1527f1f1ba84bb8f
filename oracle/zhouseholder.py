"""Plain double-complex Householder QR and the tiled algorithm in complex arithmetic.

Test infrastructure only: the CPU oracle of the double-complex tiled QR (the thesis runs
every Chapter 3 experiment in double and in double complex precision, Section 3.3).  Only
the tests, the smoke check and the benchmark's CPU legs use it; the library never imports
it and it imports nothing from the library.

Everything is unblocked and in numpy complex128: each reflector is generated and applied
on its own, in the order the mathematics gives.

Conventions (the thesis names LAPACK's kernels - the complex ones multiply by the unitary
Q, glossary entries UNMQR / TTMQR / TSMQR - but prints none of their internals; the LAPACK
complex conventions are used):
* Reflector H = I - tau v v^H with v[0] = 1.  For a vector [alpha; x]:
  beta = -sign(Re alpha) * ||[alpha; x]|| (real, sign(0) = +1), tau = (beta - alpha) / beta,
  v[1:] = x / (alpha - beta), so that H^H [alpha; x] = [beta; 0].  H = I (tau = 0) when x = 0
  and alpha is real.  The diagonal of R is therefore real.
* Q = H_1 H_2 ... H_k; the factorization applies H_j^H = I - conj(tau_j) v_j v_j^H to the
  trailing columns; Q^H C applies the H_j^H in order, Q C the H_j in reverse order.
* T factors are compact WY: H_1 ... H_b = I - V T V^H with T upper triangular, built by
  T <- [[T, -tau T V^H v], [0, tau]]; stored ib x nb per factored tile like the real case.
* Tiles, the elimination list's task program and the TS form are those of
  oracle.householder; a matrix that is not a whole number of tiles is the zero-padded one.
"""
from __future__ import annotations

import numpy as np

from .householder import tile_grid, ts_rows


def zhouseholder(alpha: complex, x: np.ndarray):
    """Reflector with H^H [alpha; x] = [beta; 0] (LAPACK ZLARFG convention, no rescaling).
    Returns (beta, tau, v_tail)."""
    alpha = complex(alpha)
    xnorm = float(np.sqrt(np.vdot(x, x).real)) if x.size else 0.0
    if xnorm == 0.0 and alpha.imag == 0.0:
        return alpha, 0j, np.zeros_like(x, dtype=np.complex128)
    norm = float(np.sqrt(abs(alpha) ** 2 + xnorm * xnorm))
    beta = -norm if alpha.real >= 0.0 else norm
    tau = (beta - alpha) / beta
    return complex(beta), tau, x / (alpha - beta)


def _apply_h_adj(tau, vv, C):
    """C <- H^H C = C - conj(tau) v (v^H C)."""
    C -= np.conj(tau) * np.outer(vv, np.conj(vv) @ C)


def _apply_h(tau, vv, C):
    """C <- H C = C - tau v (v^H C)."""
    C -= tau * np.outer(vv, np.conj(vv) @ C)


def zqr_unblocked(A: np.ndarray):
    """Householder QR of an m x n complex matrix, one column at a time.  Returns (F, tau):
    R in the upper triangle of F (real diagonal), reflectors below it."""
    F = np.array(A, dtype=np.complex128, copy=True)
    m, n = F.shape
    kmax = min(m, n)
    tau = np.zeros(kmax, dtype=np.complex128)
    for j in range(kmax):
        beta, t, v = zhouseholder(F[j, j], F[j + 1:, j])
        F[j, j] = beta
        F[j + 1:, j] = v
        tau[j] = t
        if t != 0 and j + 1 < n:
            _apply_h_adj(t, np.concatenate(([1.0 + 0j], v)), F[j:, j + 1:])
    return F, tau


def zbuild_t(V: np.ndarray, tau: np.ndarray, ib: int) -> np.ndarray:
    """Compact-WY T blocks (ib x nb layout) of reflector columns V[:, c] (full vectors)."""
    nref = V.shape[1]
    T = np.zeros((ib, len(tau)), dtype=np.complex128)
    for b0 in range(0, nref, ib):
        b1 = min(b0 + ib, nref)
        for c in range(b0, b1):
            col = c - b0
            T[col, c] = tau[c]
            if col:
                z = np.conj(V[:, b0:c]).T @ V[:, c]               # V_prev^H v
                T[:col, c] = -tau[c] * (T[:col, b0:c] @ z)
    return T


def zgeqrt(A: np.ndarray, ib: int):
    """GEQRT on one complex tile, in place.  Returns T (ib x nb)."""
    nb = A.shape[1]
    kmax = min(A.shape[0], nb)
    tau = np.zeros(nb, dtype=np.complex128)
    for j in range(kmax):
        beta, t, v = zhouseholder(A[j, j], A[j + 1:, j])
        A[j, j] = beta
        A[j + 1:, j] = v
        tau[j] = t
        if t != 0 and j + 1 < nb:
            _apply_h_adj(t, np.concatenate(([1.0 + 0j], v)), A[j:, j + 1:])
    V = np.tril(A[:, :kmax], -1) + np.eye(A.shape[0], kmax)
    T = zbuild_t(V, tau[:kmax], ib)
    if kmax < nb:
        out = np.zeros((ib, nb), dtype=np.complex128)
        out[:, :kmax] = T
        T = out
    return T


def zunmqr(V_tile, T, C, ib, adjoint=True):
    """C <- Q^H C (adjoint) or Q C with the reflectors of zgeqrt (tau = diagonal of T)."""
    k = min(V_tile.shape[0], V_tile.shape[1])
    order = range(k) if adjoint else reversed(range(k))
    for j in order:
        t = T[j % ib, j]
        if t == 0:
            continue
        vv = np.concatenate(([1.0 + 0j], V_tile[j + 1:, j]))
        (_apply_h_adj if adjoint else _apply_h)(t, vv, C[j:, :])


def _pair_reflector(c, v, t, C1, C2, rows, adjoint):
    """Apply reflector c of a TT / TS kernel (unit entry in row c of C1, tail v in rows
    'rows' of C2) to the pair [C1; C2]."""
    w = C1[c, :] + np.conj(v) @ C2[rows, :]
    f = np.conj(t) if adjoint else t
    C1[c, :] -= f * w
    C2[rows, :] -= f * np.outer(v, w)


def zttqrt(R1, A2, ib):
    """TTQRT: QR of upper triangle R1 on the upper triangle of A2 (complex), in place;
    reflector c acts on row c of R1 and rows 0..c of A2, its tail in A2[0:c+1, c]."""
    nb = R1.shape[1]
    mb = A2.shape[0]
    tau = np.zeros(nb, dtype=np.complex128)
    for c in range(nb):
        r = min(c + 1, mb)
        beta, t, v = zhouseholder(R1[c, c], A2[:r, c].copy())
        R1[c, c] = beta
        A2[:r, c] = v
        tau[c] = t
        if t != 0 and c + 1 < nb:
            _pair_reflector(c, v, t, R1[:, c + 1:], A2[:, c + 1:], slice(0, r), True)
    V = np.vstack([np.eye(nb, dtype=np.complex128), np.triu(A2[:, :nb])])
    return zbuild_t(V, tau, ib)


def ztsqrt(R1, A2, ib):
    """TSQRT: QR of upper triangle R1 on the square tile A2 (complex), in place; reflector c
    acts on row c of R1 and every row of A2, its tail overwrites A2[:, c]."""
    nb = R1.shape[1]
    tau = np.zeros(nb, dtype=np.complex128)
    for c in range(nb):
        beta, t, v = zhouseholder(R1[c, c], A2[:, c].copy())
        R1[c, c] = beta
        A2[:, c] = v
        tau[c] = t
        if t != 0 and c + 1 < nb:
            _pair_reflector(c, v, t, R1[:, c + 1:], A2[:, c + 1:], slice(None), True)
    V = np.vstack([np.eye(nb, dtype=np.complex128), A2[:, :nb]])
    return zbuild_t(V, tau, ib)


def zpair_mqr(V2, T, C1, C2, ib, ts, adjoint=True):
    """TTMQR (ts False: tails in V2's upper triangle) or TSMQR (ts True: tails fill V2):
    [C1; C2] <- Q^H [C1; C2] (adjoint) or Q [C1; C2], reflector by reflector."""
    nb = V2.shape[1]
    mb = V2.shape[0]
    order = range(nb) if adjoint else reversed(range(nb))
    for c in order:
        t = T[c % ib, c]
        if t == 0:
            continue
        rows = slice(None) if ts else slice(0, min(c + 1, mb))
        _pair_reflector(c, V2[rows, c], t, C1, C2, rows, adjoint)


def zpad(A, nb):
    m, n = A.shape
    p, q = tile_grid(m, n, nb)
    P = np.zeros((p * nb, q * nb), dtype=np.complex128)
    P[:m, :n] = A
    return P


def ztiled_qr(A: np.ndarray, nb: int, ib: int, elims, ts: bool = False):
    """Complex tiled QR following the column-by-column program of the list (TS form when
    ts): for each panel k, GEQRT(i,k) / UNMQR(i,k,j) for the rows that are triangularized,
    then each elimination of column k in list order with TT or TS kernels.  Returns
    (F, Tg, Tt) as oracle.householder.tiled_qr."""
    m, n = A.shape
    p, q = tile_grid(m, n, nb)
    F = zpad(np.asarray(A, dtype=np.complex128), nb)
    Tg = [[None] * q for _ in range(p)]
    Tt = [[None] * q for _ in range(p)]

    def tile(i, j):
        return F[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]

    by_col = {}
    for e in elims:
        by_col.setdefault(e[0], []).append(e)
    tsr = ts_rows(elims) if ts else {}
    for k in range(min(p, q)):
        sq = tsr.get(k, ())
        for i in range(k, p):
            if i in sq:
                continue
            Tg[i][k] = zgeqrt(tile(i, k), ib)
            for j in range(k + 1, q):
                zunmqr(tile(i, k), Tg[i][k], tile(i, j), ib)
        for (_, i, piv) in by_col.get(k, []):
            square = i in sq
            Tt[i][k] = (ztsqrt if square else zttqrt)(tile(piv, k), tile(i, k), ib)
            for j in range(k + 1, q):
                zpair_mqr(tile(i, k), Tt[i][k], tile(piv, j), tile(i, j), ib, square)
    return F, Tg, Tt


def zapply_q(F, Tg, Tt, nb, ib, elims, B, adjoint=True, ts=False):
    """Q^H B (adjoint) or Q B for the complex tiled factorization; B has m rows."""
    p = F.shape[0] // nb
    q = F.shape[1] // nb
    m = B.shape[0]
    Bp = np.zeros((p * nb, B.shape[1]), dtype=np.complex128)
    Bp[:m] = B

    def brow(i):
        return Bp[i * nb:(i + 1) * nb]

    def ftile(i, j):
        return F[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]

    ops = []
    by_col = {}
    for e in elims:
        by_col.setdefault(e[0], []).append(e)
    tsr = ts_rows(elims) if ts else {}
    for k in range(min(p, q)):
        sq = tsr.get(k, ())
        for i in range(k, p):
            if i not in sq:
                ops.append(("G", i, k, None))
        for (_, i, piv) in by_col.get(k, []):
            ops.append(("S" if i in sq else "T", i, k, piv))
    for kind, i, k, piv in (ops if adjoint else list(reversed(ops))):
        if kind == "G":
            zunmqr(ftile(i, k), Tg[i][k], brow(i), ib, adjoint)
        else:
            zpair_mqr(ftile(i, k), Tt[i][k], brow(piv), brow(i), ib, kind == "S", adjoint)
    return Bp[:m].copy()


def zback_substitute(R, Y):
    """Solve R X = Y for upper-triangular complex R by back substitution, row by row."""
    n = R.shape[0]
    X = np.array(Y, dtype=np.complex128, copy=True).reshape(n, -1)
    for i in reversed(range(n)):
        if i + 1 < n:
            X[i] -= R[i, i + 1:] @ X[i + 1:]
        X[i] /= R[i, i]
    return X


def zlstsq(A, B, nb, ib, elims, ts=False):
    """Complex least squares min ||A X - B||: X = R^{-1} (Q^H B)[0:n]."""
    m, n = A.shape
    F, Tg, Tt = ztiled_qr(A, nb, ib, elims, ts)
    QhB = zapply_q(F, Tg, Tt, nb, ib, elims, np.asarray(B, dtype=np.complex128).reshape(m, -1), ts=ts)
    return zback_substitute(np.triu(F[:n, :n]), QhB[:n])
