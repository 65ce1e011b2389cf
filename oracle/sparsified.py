"""CPU oracle of the sparsified-powers W pattern (Sec. 4.1, Algorithm 1) --
TEST INFRASTRUCTURE ONLY.

Initial subspace V_0 = diagonal matrices, so S = -D^{-1}(A - D) (the sign
that makes A = D (I - S) hold) and A^{-1} D = I + S + S^2 + ...  Per column
j, written out one column at a time:

    s = t = e_j
    for level = 1..k:
        t = S t                      (sum over the entries c of t, in
                                      increasing c, of S(:, c) t_c)
        drop t by count p_l          (the p_l entries of largest modulus
                                      survive, ties to the lower row; the
                                      diagonal entry j is never dropped and
                                      does not use up the count; p_l <= 0
                                      keeps everything)
        s = s + t
    structure of w_j = structure of s, optionally dropped by count to `keep`
    entries (the diagonal included) -- the fixed rule at a given nnz(W).

Entries whose sum is exactly zero are not stored.  Ordering key of an entry
v: |v|^2 = re^2 + im^2 (no square root, so both implementations compare the
same quantity).
"""
from __future__ import annotations

import numpy as np

from workloads.csc import Pattern


def _key(v) -> float:
    v = complex(v)
    return v.real * v.real + v.imag * v.imag


def _drop_by_count(vec: dict, j: int, count: int) -> dict:
    if count <= 0:
        return vec
    off = sorted((r for r in vec if r != j), key=lambda r: (-_key(vec[r]), r))
    keep = set(off[:count])
    if j in vec:
        keep.add(j)
    return {r: vec[r] for r in vec if r in keep}


def sparsified_powers(A, k: int = 2, p_l: int = 0, keep: int = 0, cols=None) -> Pattern | dict:
    """Pattern of W (all columns), or {j: sorted rows} for the listed columns."""
    n = A.n
    d = np.zeros(n, dtype=A.vals.dtype)
    for c in range(n):
        for p in range(A.colptr[c], A.colptr[c + 1]):
            if A.rowidx[p] == c:
                d[c] = A.vals[p]
    if np.any(d == 0):
        raise ValueError("sparsified powers with V_0 = diag(A) need a zero-free diagonal")
    inv = 1.0 / d

    def S_col(c):  # S(:, c) = -(1/d_i) a_ic for i != c
        for p in range(A.colptr[c], A.colptr[c + 1]):
            i = int(A.rowidx[p])
            if i != c:
                yield i, -(inv[i] * A.vals[p])

    out = {}
    for j in (range(n) if cols is None else cols):
        t = {j: A.vals.dtype.type(1)}
        s = dict(t)
        for _ in range(k):
            nt = {}
            for c in sorted(t):
                tc = t[c]
                for i, sic in S_col(c):
                    nt[i] = nt[i] + sic * tc if i in nt else sic * tc
            nt = {r: v for r, v in nt.items() if v != 0}
            t = _drop_by_count(nt, j, p_l)
            for r, v in t.items():
                s[r] = s[r] + v if r in s else v
            s = {r: v for r, v in s.items() if v != 0 or r == j}
        s = _drop_by_count(s, j, keep - 1 if keep > 0 else 0) if keep != 1 else {j: s[j]} if j in s else {}
        out[j] = sorted(s)
    if cols is not None:
        return out
    counts = np.array([len(out[j]) for j in range(n)], dtype=np.int64)
    colptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    rowidx = np.array([r for j in range(n) for r in out[j]], dtype=np.int32)
    return Pattern(n, colptr, rowidx)
