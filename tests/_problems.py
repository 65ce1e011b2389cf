"""Small seeded problems shared by the tests (input construction only)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads import CSC, Pattern


def random_sparse(n, density, seed, complex_=False, diag=3.0) -> CSC:
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csc")
    M.data = rng.standard_normal(M.data.size)
    if complex_:
        M = M.astype(np.complex128)
        M.data = M.data + 1j * rng.standard_normal(M.data.size)
    M = M + diag * sp.identity(n, format="csc")
    return CSC.from_scipy(M)


def pattern_from_sets(n, sets) -> Pattern:
    cp = np.zeros(n + 1, np.int32)
    ri = []
    for j, s in enumerate(sets):
        s = sorted(set(int(x) for x in s))
        cp[j + 1] = cp[j] + len(s)
        ri.extend(s)
    return Pattern(n, cp, np.asarray(ri, np.int32))


def pattern_from_matrix(M) -> Pattern:
    M = sp.csc_matrix(M)
    M.sort_indices()
    return Pattern(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32))


def dense(A: CSC) -> np.ndarray:
    return A.to_scipy().toarray()
