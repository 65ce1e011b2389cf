"""Compressed sparse column containers (0-based, int32 indices, sorted rows)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Pattern:
    """Sparsity structure of a standard matrix subspace: column j may be
    nonzero exactly on rowidx[colptr[j]:colptr[j+1]] (sorted ascending)."""

    n: int
    colptr: np.ndarray  # int32 [n+1]
    rowidx: np.ndarray  # int32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def col(self, j: int) -> np.ndarray:
        return self.rowidx[self.colptr[j]:self.colptr[j + 1]]

    def counts(self) -> np.ndarray:
        return np.diff(self.colptr).astype(np.int32)

    def validate(self) -> None:
        assert self.colptr.dtype == np.int32 and self.rowidx.dtype == np.int32
        assert self.colptr.shape == (self.n + 1,) and self.colptr[0] == 0
        assert np.all(np.diff(self.colptr) >= 0)
        if self.nnz:
            assert self.rowidx.min() >= 0 and self.rowidx.max() < self.n
        for j in range(self.n):
            c = self.col(j)
            assert np.all(np.diff(c) > 0), f"column {j} not strictly sorted"


@dataclass
class CSC(Pattern):
    """A square sparse matrix in CSC form; vals is float64 or complex128."""

    vals: np.ndarray = None

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.vals)

    def pattern(self) -> Pattern:
        return Pattern(self.n, self.colptr, self.rowidx)

    def to_scipy(self) -> sp.csc_matrix:
        return sp.csc_matrix((self.vals, self.rowidx, self.colptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(M) -> "CSC":
        M = sp.csc_matrix(M)
        M.sum_duplicates()
        M.sort_indices()
        vals = M.data.astype(np.complex128 if np.iscomplexobj(M.data) else np.float64)
        return CSC(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32), vals)
