"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random matrices and right-hand sides only; it contains none of the
tiled-QR arithmetic.  Haar-random orthogonal factors come from numpy's LAPACK QR of a
Gaussian matrix with the sign correction of Mezzadri (2007), so that a conditioned test
matrix A = U diag(sigma) V^T can be built.  All arrays are float64 in Fortran (column-
major) order, the layout the library takes.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1303318200  # workload seeds are SEED_BASE + 1 .. SEED_BASE + 5


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """m x n matrix of i.i.d. N(0, 1) entries."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)))


def complex_gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """m x n matrix of i.i.d. standard complex normal entries (N(0, 1/2) real and imaginary
    parts), complex128."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2.0)
    return np.asfortranarray(z)


def haar_orthonormal(m: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """m x n matrix with Haar-distributed orthonormal columns (m >= n)."""
    G = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def singular_values(n: int, cond: float) -> np.ndarray:
    """Geometrically spaced sigma_i = cond**(-(i-1)/(n-1)), i = 1..n."""
    if n == 1:
        return np.ones(1)
    return cond ** (-np.arange(n) / (n - 1))


def conditioned(m: int, n: int, cond: float, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T with Haar U (m x n), V (n x n) and geometric sigma."""
    rng = np.random.default_rng(seed)
    U = haar_orthonormal(m, n, rng)
    V = haar_orthonormal(n, n, rng)
    return np.asfortranarray((U * singular_values(n, cond)) @ V.T)


def least_squares_problem(m: int, n: int, cond: float, noise: float, nrhs: int, seed: int):
    """(A, X, B): conditioned A, X ~ N(0,1) (n x nrhs), B = A X + noise * N(0,1)."""
    A = conditioned(m, n, cond, seed)
    rng = np.random.default_rng(seed + 7919)
    X = rng.standard_normal((n, nrhs))
    B = A @ X + noise * rng.standard_normal((m, nrhs))
    return A, np.asfortranarray(X), np.asfortranarray(B)


def ragged_batch_shapes(count: int, seed: int, m_lo: int = 256, m_hi: int = 8192,
                        n_choices=(32, 64, 128, 256)):
    """Shapes of a batch of tall matrices: rows uniform in [m_lo, m_hi], columns
    uniform in n_choices (never more columns than rows)."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = rng.choice(np.asarray(n_choices), size=count)
    return [(int(m), int(min(n, m))) for m, n in zip(ms, ns)]


def conditioned_device(m: int, n: int, cond: float, seed: int, device):
    """Device-side (torch) version of conditioned() for inputs too large to build on the
    host: A = U diag(sigma) V^T, U (m x n) and V (n x n) Haar from the QR of seeded
    Gaussians with Mezzadri's sign correction.  Returned as a column-major float64 CUDA
    tensor (stride (1, m)).  Deterministic for a given seed and device type."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def haar(rows, cols):
        G = torch.randn(rows, cols, dtype=torch.float64, device=device, generator=g)
        Q, R = torch.linalg.qr(G)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d

    U = haar(m, n)
    V = haar(n, n)
    sig = torch.from_numpy(singular_values(n, cond)).to(device)
    A = (U * sig) @ V.T
    return A.t().contiguous().t()


def least_squares_device(m: int, n: int, cond: float, noise: float, nrhs: int, seed: int, device):
    """(A, X, B) of least_squares_problem() built on the device (see conditioned_device)."""
    import torch
    A = conditioned_device(m, n, cond, seed, device)
    g = torch.Generator(device=device)
    g.manual_seed(seed + 7919)
    X = torch.randn(n, nrhs, dtype=torch.float64, device=device, generator=g)
    B = A @ X + noise * torch.randn(m, nrhs, dtype=torch.float64, device=device, generator=g)
    return A, X.t().contiguous().t(), B.t().contiguous().t()
