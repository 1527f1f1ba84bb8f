"""FP64 least-squares quality measures used to judge every solver against the oracle.

Test infrastructure only (see the package docstring).

For min ||A x - b||, the residual r = b - A x of the exact solution satisfies
A^T r = 0, so ||A^T r|| / (||A||_F ||r||) measures how far a computed x is from being a
least-squares solution (a normwise backward-error proxy, Higham, 'Accuracy and Stability
of Numerical Algorithms', 2nd ed., Section 20.7).
"""
from __future__ import annotations

import numpy as np


def residual(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    return np.asarray(B, dtype=np.float64) - np.asarray(A, dtype=np.float64) @ X


def ls_optimality(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> float:
    """max over right-hand sides of ||A^T r_j|| / (||A||_F ||r_j||)."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[1], -1)
    R = residual(A, X, np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1))
    AtR = A.T @ R
    na = np.linalg.norm(A)
    out = 0.0
    for j in range(R.shape[1]):
        nr = np.linalg.norm(R[:, j])
        out = max(out, np.linalg.norm(AtR[:, j]) / (na * nr) if nr > 0 else 0.0)
    return out


def rel_error(X: np.ndarray, Xref: np.ndarray) -> float:
    """||X - Xref||_F / ||Xref||_F."""
    return float(np.linalg.norm(np.asarray(X) - np.asarray(Xref)) / np.linalg.norm(Xref))
