"""Plain FP64 Householder QR, the tiled TT / TS algorithms, apply-Q and least squares.

Test infrastructure only: the CPU oracle for the numeric side of tiled QR.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it; the library
never imports it and it imports nothing from the library.

Everything here is deliberately unblocked: each reflector is generated and applied on
its own, in the order the mathematics gives, in numpy float64.

Conventions (the thesis names LAPACK's kernels but prints none of their internals; the
LAPACK conventions are used, Section 1.3 and Section 3.1.1):
* Reflector H = I - tau v v^T with v[0] = 1 (implicit).  For a vector [alpha; x]:
  beta = -sign(alpha) * ||[alpha; x]|| with sign(0) = +1, tau = (beta - alpha)/beta,
  v[1:] = x / (alpha - beta); tau = 0 and H = I when ||x|| = 0.
* A factored tile keeps R in its upper triangle and the GEQRT reflectors below the
  diagonal (unit diagonal implicit).  TTQRT stores its reflectors in the upper triangle
  of the zeroed tile: reflector c lives in rows 0..c of column c.  TSQRT zeroes a
  square tile and stores reflector c in the whole column c of that tile.
* T factors are compact-WY (Schreiber-Van Loan): for each block of ib reflectors,
  H_1 ... H_b = I - V T V^T with T upper triangular, built by
  T <- [[T, -tau T V^T v], [0, tau]].  One factored tile stores its T blocks side by
  side in an ib x nb array (block b in columns b*ib .. b*ib+ib-1), like LAPACK GEQRT.
* A matrix that is not a whole number of tiles is processed as the zero-padded
  p*nb x q*nb matrix (p = ceil(m/nb), q = ceil(n/nb)); zero rows and columns leave the
  leading R, V and T unchanged.
"""
from __future__ import annotations

import numpy as np


def householder(alpha: float, x: np.ndarray):
    """Reflector annihilating x below alpha (LAPACK DLARFG convention, no rescaling).
    Returns (beta, tau, v_tail)."""
    xnorm = float(np.sqrt(np.dot(x, x))) if x.size else 0.0
    if xnorm == 0.0:
        return alpha, 0.0, np.zeros_like(x)
    norm = float(np.sqrt(alpha * alpha + xnorm * xnorm))
    beta = -norm if alpha >= 0.0 else norm
    tau = (beta - alpha) / beta
    return beta, tau, x / (alpha - beta)


# ---------------------------------------------------------------------------
# Unblocked Householder QR of a whole matrix (Golub-Van Loan Algorithm 5.2.1 form)
# ---------------------------------------------------------------------------

def qr_unblocked(A: np.ndarray):
    """Householder QR of an m x n matrix, one column at a time.  Returns (F, tau):
    R in the upper triangle of F, reflectors below it."""
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    kmax = min(m, n)
    tau = np.zeros(kmax)
    for j in range(kmax):
        beta, t, v = householder(F[j, j], F[j + 1:, j])
        F[j, j] = beta
        F[j + 1:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < n:
            vv = np.concatenate(([1.0], v))
            w = vv @ F[j:, j + 1:]
            F[j:, j + 1:] -= t * np.outer(vv, w)
    return F, tau


def form_q(F: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Explicit m x m Q = H_0 H_1 ... H_{k-1} of qr_unblocked's output."""
    m = F.shape[0]
    Q = np.eye(m)
    for j in reversed(range(len(tau))):
        vv = np.concatenate(([1.0], F[j + 1:, j]))
        Q[j:, :] -= tau[j] * np.outer(vv, vv @ Q[j:, :])
    return Q


# ---------------------------------------------------------------------------
# Compact-WY T (Schreiber-Van Loan)
# ---------------------------------------------------------------------------

def build_t(V: np.ndarray, tau: np.ndarray, ib: int) -> np.ndarray:
    """T blocks for reflector columns V[:, c] (full vectors, unit entries included),
    laid out ib x nb: block b holds reflectors b*ib .. in its columns."""
    nref = V.shape[1]
    nb = len(tau)
    T = np.zeros((ib, nb))
    for b0 in range(0, nref, ib):
        b1 = min(b0 + ib, nref)
        for c in range(b0, b1):
            col = c - b0
            T[col, c] = tau[c]
            if col:
                z = V[:, b0:c].T @ V[:, c]                     # V_prev^T v
                T[:col, c] = -tau[c] * (T[:col, b0:c] @ z)    # -tau T_prev (V^T v)
    return T


# ---------------------------------------------------------------------------
# The four tile kernels (Table 'Kernels for tiled QR'), one reflector at a time
# ---------------------------------------------------------------------------

def geqrt(A: np.ndarray, ib: int):
    """GEQRT on one nb x nb tile, in place.  Returns T (ib x nb)."""
    nb = A.shape[1]
    kmax = min(A.shape[0], nb)
    tau = np.zeros(nb)
    for j in range(kmax):
        beta, t, v = householder(A[j, j], A[j + 1:, j])
        A[j, j] = beta
        A[j + 1:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < nb:
            vv = np.concatenate(([1.0], v))
            w = vv @ A[j:, j + 1:]
            A[j:, j + 1:] -= t * np.outer(vv, w)
    V = np.tril(A[:, :kmax], -1) + np.eye(A.shape[0], kmax)
    return build_t(V, tau[:kmax], ib) if kmax == nb else _pad_t(build_t(V, tau[:kmax], ib), nb)


def _pad_t(T, nb):
    out = np.zeros((T.shape[0], nb))
    out[:, :T.shape[1]] = T
    return out


def unmqr(V_tile: np.ndarray, T: np.ndarray, C: np.ndarray, ib: int):
    """UNMQR: C <- Q^T C with Q from GEQRT of V_tile; applied reflector by reflector
    (tau is read from the diagonal of each T block)."""
    nb = V_tile.shape[1]
    for j in range(min(V_tile.shape[0], nb)):
        t = T[j % ib, j]
        if t == 0.0:
            continue
        vv = np.concatenate(([1.0], V_tile[j + 1:, j]))
        C[j:, :] -= t * np.outer(vv, vv @ C[j:, :])


def ttqrt(R1: np.ndarray, A2: np.ndarray, ib: int):
    """TTQRT: QR of the upper triangle R1 stacked on the upper triangle of A2, in place.
    Reflector c acts on row c of R1 and rows 0..c of A2; its tail is stored in
    A2[0:c+1, c].  Returns T (ib x nb)."""
    nb = R1.shape[1]
    mb = A2.shape[0]
    tau = np.zeros(nb)
    for c in range(nb):
        r = min(c + 1, mb)
        beta, t, v = householder(R1[c, c], A2[:r, c].copy())
        R1[c, c] = beta
        A2[:r, c] = v
        tau[c] = t
        if t != 0.0 and c + 1 < nb:
            w = R1[c, c + 1:] + v @ A2[:r, c + 1:]
            R1[c, c + 1:] -= t * w
            A2[:r, c + 1:] -= t * np.outer(v, w)
    # the implicit reflectors: unit entry in R1's row c, tail in A2's upper triangle
    V = np.vstack([np.eye(nb), np.triu(A2[:, :nb])])
    return build_t(V, tau, ib)


def ttmqr(V2: np.ndarray, T: np.ndarray, C1: np.ndarray, C2: np.ndarray, ib: int):
    """TTMQR: [C1; C2] <- Q^T [C1; C2] with Q from TTQRT (reflectors in the upper
    triangle of V2), applied reflector by reflector."""
    nb = V2.shape[1]
    mb = V2.shape[0]
    for c in range(nb):
        t = T[c % ib, c]
        if t == 0.0:
            continue
        r = min(c + 1, mb)
        v = V2[:r, c]
        w = C1[c, :] + v @ C2[:r, :]
        C1[c, :] -= t * w
        C2[:r, :] -= t * np.outer(v, w)


def tsqrt(R1: np.ndarray, A2: np.ndarray, ib: int):
    """TSQRT: QR of the upper triangle R1 stacked on the square tile A2, in place
    (Algorithm 'elimSQ').  Reflector c acts on row c of R1 and on every row of A2; its
    tail overwrites column c of A2.  Returns T (ib x nb)."""
    nb = R1.shape[1]
    tau = np.zeros(nb)
    for c in range(nb):
        beta, t, v = householder(R1[c, c], A2[:, c].copy())
        R1[c, c] = beta
        A2[:, c] = v
        tau[c] = t
        if t != 0.0 and c + 1 < nb:
            w = R1[c, c + 1:] + v @ A2[:, c + 1:]
            R1[c, c + 1:] -= t * w
            A2[:, c + 1:] -= t * np.outer(v, w)
    # the implicit reflectors: unit entry in R1's row c, tail in A2's column c
    V = np.vstack([np.eye(nb), A2[:, :nb]])
    return build_t(V, tau, ib)


def tsmqr(V2: np.ndarray, T: np.ndarray, C1: np.ndarray, C2: np.ndarray, ib: int):
    """TSMQR: [C1; C2] <- Q^T [C1; C2] with Q from TSQRT (reflector c's tail is the
    whole column c of V2), applied reflector by reflector."""
    nb = V2.shape[1]
    for c in range(nb):
        t = T[c % ib, c]
        if t == 0.0:
            continue
        v = V2[:, c]
        w = C1[c, :] + v @ C2
        C1[c, :] -= t * w
        C2 -= t * np.outer(v, w)


def _apply_ts_reflectors_reversed(V2, T, C1, C2, ib):
    nb = V2.shape[1]
    for c in reversed(range(nb)):
        t = T[c % ib, c]
        if t == 0.0:
            continue
        v = V2[:, c]
        w = C1[c, :] + v @ C2
        C1[c, :] -= t * w
        C2 -= t * np.outer(v, w)


def ts_rows(elims):
    """Rows each column zeroes with TS kernels in the TS form of a list: the rows that
    are never a pivot in that column (a TS elimination needs a square, not yet
    triangularized, tile; every pivot was triangularized by GEQRT)."""
    piv_rows = {}
    for (k, _, piv) in elims:
        piv_rows.setdefault(k, set()).add(piv)
    out = {}
    for (k, i, _) in elims:
        if i not in piv_rows.get(k, ()):
            out.setdefault(k, set()).add(i)
    return out


# ---------------------------------------------------------------------------
# The tiled TT algorithm driven by an elimination list (Algorithm 'elimTR')
# ---------------------------------------------------------------------------

def tile_grid(m: int, n: int, nb: int):
    return -(-m // nb), -(-n // nb)


def pad(A: np.ndarray, nb: int) -> np.ndarray:
    m, n = A.shape
    p, q = tile_grid(m, n, nb)
    P = np.zeros((p * nb, q * nb))
    P[:m, :n] = A
    return P


def tiled_qr(A: np.ndarray, nb: int, ib: int, elims, ts: bool = False):
    """Tiled QR of A (m x n) following the column-by-column program: for each panel k,
    GEQRT(i,k) and UNMQR(i,k,j) for every row i >= k, then TTQRT(i,piv,k) and
    TTMQR(i,piv,k,j) for each elimination of column k in list order.

    ts: the TS form of the list - rows that are never a pivot in column k skip GEQRT /
    UNMQR there and are zeroed by TSQRT(i,piv,k) / TSMQR(i,piv,k,j) instead (Algorithm
    'elimSQ'); the other eliminations stay TT.

    Returns (F, Tg, Tt): F is the factored zero-padded matrix (p*nb x q*nb); Tg[i][k]
    and Tt[i][k] are the ib x nb T factors of GEQRT(i,k) and of the TTQRT or TSQRT that
    zeroed tile (i,k) (None where the kernel did not run)."""
    m, n = A.shape
    p, q = tile_grid(m, n, nb)
    F = pad(np.asarray(A, dtype=np.float64), nb)
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
            Tg[i][k] = geqrt(tile(i, k), ib)
            for j in range(k + 1, q):
                unmqr(tile(i, k), Tg[i][k], tile(i, j), ib)
        for (_, i, piv) in by_col.get(k, []):
            if i in sq:
                Tt[i][k] = tsqrt(tile(piv, k), tile(i, k), ib)
                for j in range(k + 1, q):
                    tsmqr(tile(i, k), Tt[i][k], tile(piv, j), tile(i, j), ib)
            else:
                Tt[i][k] = ttqrt(tile(piv, k), tile(i, k), ib)
                for j in range(k + 1, q):
                    ttmqr(tile(i, k), Tt[i][k], tile(piv, j), tile(i, j), ib)
    return F, Tg, Tt


def apply_qt(F: np.ndarray, Tg, Tt, nb: int, ib: int, elims, B: np.ndarray,
             transpose: bool = True, ts: bool = False) -> np.ndarray:
    """Q^T B (transpose=True) or Q B for the tiled factorization; B has m rows.  Q^T
    replays the update kernels on B's tile rows in program order; Q applies the same
    reflectors in the reverse order.  ts: the factorization used the TS form."""
    p = F.shape[0] // nb
    q = F.shape[1] // nb
    m = B.shape[0]
    Bp = np.zeros((p * nb, B.shape[1]))
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
    if transpose:
        for kind, i, k, piv in ops:
            if kind == "G":
                unmqr(ftile(i, k), Tg[i][k], brow(i), ib)
            elif kind == "S":
                tsmqr(ftile(i, k), Tt[i][k], brow(piv), brow(i), ib)
            else:
                ttmqr(ftile(i, k), Tt[i][k], brow(piv), brow(i), ib)
    else:
        for kind, i, k, piv in reversed(ops):
            if kind == "G":
                _apply_geqrt_reflectors_reversed(ftile(i, k), Tg[i][k], brow(i), ib)
            elif kind == "S":
                _apply_ts_reflectors_reversed(ftile(i, k), Tt[i][k], brow(piv), brow(i), ib)
            else:
                _apply_tt_reflectors_reversed(ftile(i, k), Tt[i][k], brow(piv), brow(i), ib)
    return Bp[:m].copy()


def _apply_geqrt_reflectors_reversed(V_tile, T, C, ib):
    nb = V_tile.shape[1]
    for j in reversed(range(min(V_tile.shape[0], nb))):
        t = T[j % ib, j]
        if t == 0.0:
            continue
        vv = np.concatenate(([1.0], V_tile[j + 1:, j]))
        C[j:, :] -= t * np.outer(vv, vv @ C[j:, :])


def _apply_tt_reflectors_reversed(V2, T, C1, C2, ib):
    nb = V2.shape[1]
    mb = V2.shape[0]
    for c in reversed(range(nb)):
        t = T[c % ib, c]
        if t == 0.0:
            continue
        r = min(c + 1, mb)
        v = V2[:r, c]
        w = C1[c, :] + v @ C2[:r, :]
        C1[c, :] -= t * w
        C2[:r, :] -= t * np.outer(v, w)


def r_factor(F: np.ndarray, n: int) -> np.ndarray:
    """The n x n upper-triangular R of a factored matrix (m >= n)."""
    return np.triu(F[:n, :n])


def back_substitute(R: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Solve R X = Y for upper-triangular R by back substitution, row by row."""
    n = R.shape[0]
    X = np.array(Y, dtype=np.float64, copy=True).reshape(n, -1)
    for i in reversed(range(n)):
        if i + 1 < n:
            X[i] -= R[i, i + 1:] @ X[i + 1:]
        X[i] /= R[i, i]
    return X


def lstsq(A: np.ndarray, B: np.ndarray, nb: int, ib: int, elims, ts: bool = False) -> np.ndarray:
    """Least-squares solution of min ||A X - B|| (m >= n, full rank):
    X = R^{-1} (Q^T B)[0:n]."""
    m, n = A.shape
    F, Tg, Tt = tiled_qr(A, nb, ib, elims, ts)
    QtB = apply_qt(F, Tg, Tt, nb, ib, elims, np.asarray(B, dtype=np.float64).reshape(m, -1), ts=ts)
    return back_substitute(r_factor(F, n), QtB[:n])
