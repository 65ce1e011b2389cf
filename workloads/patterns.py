"""Symbolic sparsity patterns (standard matrix subspaces, Sec. 2 and Sec. 4.2).

Only structure is computed here (boolean products), no values: the W
pattern pattern(A^p) and the per-column budgets of the Gauss-Seidel V
structure (Definition in Sec. 4.2: the diagonal plus the strictly upper, or
lower, triangle of pattern(A)).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .csc import CSC, Pattern


def pattern_of(M) -> Pattern:
    if isinstance(M, CSC):
        return M.pattern()
    M = sp.csc_matrix(M)
    M.sort_indices()
    return Pattern(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32))


def _bool(A: CSC) -> sp.csc_matrix:
    return sp.csc_matrix((np.ones(A.nnz, dtype=np.float64), A.rowidx, A.colptr), shape=(A.n, A.n))


def pattern_power(A: CSC | Pattern, p: int) -> Pattern:
    """Structure of A^p (structural product: no cancellation is assumed)."""
    B = _bool(A)
    P = B.copy()
    for _ in range(p - 1):
        P = (P @ B).tocsc()
        P.data[:] = 1.0
    P.sort_indices()
    return Pattern(A.n, P.indptr.astype(np.int32), P.indices.astype(np.int32))


def upper_budget(A: CSC | Pattern) -> np.ndarray:
    """l_j budget of the upper Gauss-Seidel structure: #{i <= j : A_ij != 0},
    the diagonal counted (at least 1)."""
    col = np.repeat(np.arange(A.n), np.diff(A.colptr))
    cnt = np.bincount(col[A.rowidx < col], minlength=A.n) + 1
    return cnt.astype(np.int32)


def lower_budget(A: CSC | Pattern) -> np.ndarray:
    col = np.repeat(np.arange(A.n), np.diff(A.colptr))
    cnt = np.bincount(col[A.rowidx > col], minlength=A.n) + 1
    return cnt.astype(np.int32)


def diagonal_pattern(n: int) -> Pattern:
    return Pattern(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32))


def gauss_seidel_upper(A: CSC | Pattern) -> Pattern:
    """Fixed V structure: diagonal plus strictly upper part of pattern(A)."""
    col = np.repeat(np.arange(A.n), np.diff(A.colptr))
    keep = A.rowidx < col
    r = np.concatenate([A.rowidx[keep], np.arange(A.n)])
    c = np.concatenate([col[keep], np.arange(A.n)])
    M = sp.csc_matrix((np.ones(r.size), (r, c)), shape=(A.n, A.n))
    M.sort_indices()
    return Pattern(A.n, M.indptr.astype(np.int32), M.indices.astype(np.int32))

