"""The seeded synthetic inputs: sizes of the five configurations (the recipe's
numbers: n, nnz(A), nnz of the W pattern), determinism of the generators, and
the structural properties the method relies on (sorted rows, a full diagonal,
the upper budget's bounds).  CPU only."""
import numpy as np
import pytest

from workloads import make_workload

SIZES = {  # name: (n, nnz(A), nnz(PW), complex)
    "convdiff32": (1024, 4992, 4992, False),
    "convdiff256_A2": (65536, 326656, 846852, False),
    "powerlaw200k": (200000, 1460251, 1460251, False),
    "helmholtz512": (262144, 2353156, 2353156, True),
    "lognormal64": (262144, 1810432, 6382336, False),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_sizes(name):
    n, nnz_a, nnz_w, cplx = SIZES[name]
    w = make_workload(name)
    assert w.n == n and len(w.A.rowidx) == nnz_a and len(w.PW.rowidx) == nnz_w
    assert w.A.is_complex == cplx
    assert w.budget is None or (len(w.budget) == n and np.all(w.budget >= 1))


@pytest.mark.parametrize("name", ["convdiff32", "powerlaw200k", "lognormal64"])
def test_generators_are_deterministic(name):
    a, b = make_workload(name), make_workload(name)
    assert np.array_equal(a.A.colptr, b.A.colptr) and np.array_equal(a.A.rowidx, b.A.rowidx)
    assert np.array_equal(a.A.vals, b.A.vals) and np.array_equal(a.PW.rowidx, b.PW.rowidx)


@pytest.mark.parametrize("name", sorted(SIZES))
def test_structure(name):
    w = make_workload(name)
    for M in (w.A, w.PW):
        cp, ri = np.asarray(M.colptr), np.asarray(M.rowidx)
        assert cp[0] == 0 and np.all(np.diff(cp) >= 0) and cp[-1] == ri.size
        assert ri.min() >= 0 and ri.max() < w.n
        # rows sorted and unique within every column
        col = np.repeat(np.arange(w.n), np.diff(cp))
        key = col.astype(np.int64) * w.n + ri
        assert np.all(np.diff(key) > 0)
    # every column of A holds its diagonal entry, nonzero
    cp, ri, v = np.asarray(w.A.colptr), np.asarray(w.A.rowidx), np.asarray(w.A.vals)
    col = np.repeat(np.arange(w.n), np.diff(cp))
    d = ri == col
    assert np.count_nonzero(d) == w.n and np.all(v[d] != 0)
