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


def _keep_top(M: sp.csc_matrix, count: int) -> sp.csc_matrix:
    """Numerical dropping by count (Sec. 4.1): per column the `count` entries
    of largest magnitude survive, ties to the lower row; the diagonal is not
    subject to dropping and does not use up the count.  count < 0 keeps all."""
    M = sp.csc_matrix(M)
    M.sort_indices()
    if count < 0:
        return M
    n = M.shape[0]
    col = np.repeat(np.arange(n), np.diff(M.indptr))
    diag = M.indices == col
    order = np.lexsort((M.indices, -np.abs(M.data), col))  # by column, |value| desc, row
    rank = np.empty(order.size, dtype=np.int64)
    starts = M.indptr[:-1]
    # rank among the off-diagonal entries of its column
    od = ~diag[order]
    csum = np.cumsum(od)
    first = np.concatenate([[0], csum])[starts[col[order]]]
    rank[order] = csum - first - 1
    keep = diag | (rank < count)
    K = sp.csc_matrix((M.data[keep], M.indices[keep], np.concatenate([[0], np.cumsum(
        np.bincount(col[keep], minlength=n))])), shape=M.shape)
    K.sort_indices()
    return K


def neumann_pattern(A: CSC, k: int = 2, p_l: int = 0, keep: int = 0) -> Pattern:
    """W structure by sparsified powers (Algorithm 3 of Sec. 4.1) with the
    diagonal initial subspace V_0 = diag(A): S = -D^{-1}(A - D), so that
    A = D (I - S) and A^{-1} D = I + S + S^2 + ...; per column s_j = e_j +
    t_1 + ... + t_k with t_l = S t_{l-1} (t_0 = e_j) dropped by count p_l.
    `keep` > 0 then drops s_j itself by count to `keep` entries, the diagonal
    included (the fixed rule at a given nnz(W) per column)."""
    M = A.to_scipy()
    d = M.diagonal()
    if np.any(d == 0):
        raise ValueError("sparsified powers with V_0 = diag(A) need a zero-free diagonal")
    Dinv = sp.diags(1.0 / d)
    S = (-(Dinv @ (M - sp.diags(d)))).tocsc()
    t = sp.identity(A.n, dtype=M.dtype, format="csc")
    s = t.copy()
    for _ in range(k):
        t = _keep_top(S @ t, p_l if p_l > 0 else -1)
        s = (s + t).tocsc()
    s = _keep_top(s, keep - 1 if keep > 0 else -1)
    s.sort_indices()
    return Pattern(A.n, s.indptr.astype(np.int32), s.indices.astype(np.int32))
