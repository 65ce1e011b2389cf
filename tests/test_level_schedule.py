"""The apply's level schedule (diaf_level_schedule: host code of the library,
no GPU needed) against a brute-force longest-path computation, and its
structure checks."""
import numpy as np
import pytest
import scipy.sparse as sp

from tests._problems import pattern_from_sets


@pytest.fixture(scope="module")
def D():
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


def brute_levels(M):
    """level[i] = longest dependency chain below row i, by repeated relaxation (dense, small n)."""
    n = M.shape[0]
    Md = M.toarray() != 0
    lev = np.zeros(n, dtype=np.int64)
    for _ in range(n + 1):
        new = lev.copy()
        for i in range(n):
            deps = [j for j in range(n) if j != i and Md[i, j]]
            new[i] = max([lev[j] + 1 for j in deps], default=0)
        if np.array_equal(new, lev):
            break
        lev = new
    return lev


def csc(M):
    M = sp.csc_matrix(M)
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32)


@pytest.mark.parametrize("upper", [True, False])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_levels_match_brute_force(D, upper, seed):
    rng = np.random.default_rng(seed)
    n = 40
    M = sp.random(n, n, density=0.08, random_state=rng, format="csr")
    M = (sp.triu(M, 1) if upper else sp.tril(M, -1)) + sp.identity(n)
    cp, ri = csc(M)
    lev, nlev, up = D.level_schedule(cp, ri)
    want = brute_levels(M)
    assert np.array_equal(lev, want) and nlev == want.max() + 1
    assert up == upper or not (sp.triu(M, 1).nnz or sp.tril(M, -1).nnz)


def test_bidiagonal_and_diagonal(D):
    n = 9
    up = sp.identity(n) + sp.diags([np.ones(n - 1)], [1])
    lev, nlev, is_up = D.level_schedule(*csc(up))
    assert is_up and nlev == n and list(lev) == list(range(n - 1, -1, -1))  # t_{n-1} first
    lo = sp.identity(n) + sp.diags([np.ones(n - 1)], [-1])
    lev, nlev, is_up = D.level_schedule(*csc(lo))
    assert not is_up and nlev == n and list(lev) == list(range(n))
    lev, nlev, is_up = D.level_schedule(*csc(sp.identity(n)))
    assert nlev == 1 and not lev.any()


def test_rows_in_any_order_within_a_column(D):
    n = 6
    M = sp.identity(n) + sp.diags([np.ones(n - 2)], [2])
    cp, ri = csc(M)
    for j in range(n):  # reverse each column's rows
        ri[cp[j]:cp[j + 1]] = ri[cp[j]:cp[j + 1]][::-1]
    lev, nlev, _ = D.level_schedule(cp, ri)
    assert np.array_equal(lev, brute_levels(M))


def test_structure_errors(D):
    n = 8
    tri = pattern_from_sets(n, [[r for r in (j - 1, j, j + 1) if 0 <= r < n] for j in range(n)])
    with pytest.raises(D.DiafError) as e:
        D.level_schedule(tri.colptr, tri.rowidx)
    assert e.value.status == D.DIAF_EINVAL and "triangular" in str(e.value)
    nodiag = pattern_from_sets(n, [[j] if j != 3 else [2] for j in range(n)])
    with pytest.raises(D.DiafError) as e:
        D.level_schedule(nodiag.colptr, nodiag.rowidx)
    assert "diagonal" in str(e.value)
    bad = pattern_from_sets(n, [[j] for j in range(n)])
    ri = bad.rowidx.copy()
    ri[2] = 99
    with pytest.raises(D.DiafError) as e:
        D.level_schedule(bad.colptr, ri)
    assert "out of range" in str(e.value)
    lev, nlev, up = D.level_schedule(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert nlev == 0 and lev.size == 0


def rowwise_levels(cp, ri, n, upper):
    """Depth of every row from V's rows (the transpose of the columns the
    library walks): rows in the solve's order, each one level below the
    deepest row it reads."""
    M = sp.csc_matrix((np.ones(len(ri)), ri, cp), shape=(n, n)).tocsr()
    lev = np.zeros(n, dtype=np.int64)
    order = range(n - 1, -1, -1) if upper else range(n)
    for i in order:
        deps = [j for j in M.indices[M.indptr[i]:M.indptr[i + 1]] if j != i]
        lev[i] = max((lev[j] + 1 for j in deps), default=0)
    return lev


@pytest.mark.parametrize("name,lower", [("convdiff32", False), ("helmholtz40", False), ("convdiff32", True)])
def test_levels_of_the_oracles_v(D, name, lower):
    """The V the method builds on a workload (the oracle's, upper or lower
    rule): the library's walk against the row-wise depths."""
    import oracle as O
    from workloads import lower_budget, make_workload
    w = make_workload(name)
    rule, budget = (O.RULE_LOWER, lower_budget(w.A)) if lower else (w.vrule, w.budget)
    o = O.factor(w.A, w.PW, rule, budget, alg="S", tie_tol=w.tie_tol)
    cp = np.ascontiguousarray(o.voff, np.int32)
    ri = np.ascontiguousarray(o.Vrowidx, np.int32)
    lev, nlev, up = D.level_schedule(cp, ri)
    want = rowwise_levels(cp, ri, w.n, not lower)
    assert bool(up) == (not lower)
    assert np.array_equal(lev, want) and nlev == want.max() + 1
