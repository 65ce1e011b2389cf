"""CUDA path against the CPU oracle, element by element, through the C ABI.

Small workloads (several tiles, ragged tails, boundary columns) are compared
on every column; the full-size 256 x 256 convection-diffusion workload with
W = pattern(A^2) is compared on every column too (the oracle takes about a
second there).  Edge cases: empty matrix, empty W columns, fixed V patterns,
the lower rule, the diagonal-only (sparse approximate inverse) V.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from tests._parity import assert_parity, compare, host_factors
from tests._problems import pattern_from_sets, random_sparse
from workloads import diagonal_pattern, make_workload, pattern_of, pattern_power, upper_budget

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


def run_gpu(D, A, PW, vrule=O.RULE_UPPER, budget=None, Vfixed=None, alg="S", prec="fp64", tie_tol=O.TIE_TOL,
            stab_tol=0.0):
    dA = D.DeviceCSC.from_host(A)
    dP = D.DeviceCSC.from_host(PW)
    dB = None if budget is None else torch.from_numpy(np.ascontiguousarray(budget, np.int32)).cuda()
    dV = None if Vfixed is None else D.DeviceCSC.from_host(Vfixed)
    F = D.factor(dA, dP, vrule, dB, dV, alg=alg, prec=prec, tie_tol=tie_tol, stab_tol=stab_tol)
    torch.cuda.synchronize()
    return F


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name", ["convdiff32", "convdiff48_A2", "helmholtz40", "lognormal16", "powerlaw6k"])
def test_parity_workloads(D, name, alg):
    w = make_workload(name)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    assert np.array_equal(g["Vcp"], o.voff.astype(np.int32))
    rep = compare(g, o, w.A, w.PW, alg)
    assert_parity(rep)


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_parity_full_size_convdiff256(D, alg):
    """Full 65,536-column workload in the launch configuration the benchmark uses."""
    w = make_workload("convdiff256_A2")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    rep = compare(g, o, w.A, w.PW, alg)
    assert_parity(rep)


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("cplx", [False, True])
def test_parity_random_fixed_and_rules(D, alg, cplx):
    A = random_sparse(300, 0.015, 17, cplx)
    PW = pattern_of(A)
    for vrule, budget, Vf in ((O.RULE_UPPER, upper_budget(A), None), (O.RULE_LOWER, None, None),
                              (O.RULE_ALL, np.full(A.n, 4, np.int32), None),
                              (O.RULE_FIXED, None, diagonal_pattern(A.n)),
                              (O.RULE_FIXED, None, pattern_of(sp.triu(A.to_scipy())))):
        F = run_gpu(D, A, PW, vrule, budget, Vf, alg=alg)
        g = host_factors(F)
        o = O.factor(A, PW, vrule, budget, Vf, alg=alg)
        rep = compare(g, o, A, PW, alg)
        assert_parity(rep)


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_parity_full_size_powerlaw_sampled(D, alg):
    """n = 200,000 with tiles up to 626 x 60 in all three size buckets: every
    column of the largest bucket plus a seeded sample of the others."""
    w = make_workload("powerlaw200k")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    g = host_factors(F)
    k = w.PW.counts()
    nnz = np.diff(w.A.colptr)
    E = np.bincount(np.repeat(np.arange(w.n), k), weights=nnz[w.PW.rowidx], minlength=w.n)
    big = np.nonzero((k > 32) | (E > 200))[0]
    rng = np.random.default_rng(3)
    cols = np.unique(np.concatenate([big[:1500], rng.choice(w.n, 1500, replace=False)])).astype(np.int32)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol, cols=cols)
    rep = compare(g, o, w.A, w.PW, alg, cols=cols)
    assert_parity(rep)
    assert F.info.bucket_cols[2] > 0


def test_empty_matrix(D):
    from workloads import CSC, Pattern
    A = CSC(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    P = Pattern(0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    F = run_gpu(D, A, P, O.RULE_UPPER, None)
    assert F.n == 0 and F.V.nnz == 0


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_empty_w_columns(D, alg):
    A = random_sparse(64, 0.05, 4)
    sets = [A.col(j) for j in range(A.n)]
    for j in (0, 5, 63):
        sets[j] = []
    PW = pattern_from_sets(A.n, sets)
    F = run_gpu(D, A, PW, O.RULE_UPPER, upper_budget(A), alg=alg)
    g = host_factors(F)
    o = O.factor(A, PW, O.RULE_UPPER, upper_budget(A), alg=alg)
    assert_parity(compare(g, o, A, PW, alg))
    assert all(g["flags"][j] & 32 for j in (0, 5, 63))


def test_invalid_indices_rejected(D):
    A = random_sparse(16, 0.2, 2)
    PW = pattern_of(A)
    bad = type(PW)(PW.n, PW.colptr.copy(), PW.rowidx.copy())
    bad.rowidx[3] = 99  # out of range
    with pytest.raises(D.DiafError) as e:
        run_gpu(D, A, bad)
    assert e.value.status == D.DIAF_EINVAL


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name", ["convdiff32", "helmholtz40"])
def test_apply_matches_oracle(D, name, alg):
    w = make_workload(name)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg)
    M = O.Preconditioner(o.W_csc(), o.V_csc())
    rng = np.random.default_rng(0)
    x = rng.standard_normal(w.n) + (1j * rng.standard_normal(w.n) if w.A.is_complex else 0)
    y = F.apply(torch.from_numpy(x).cuda())
    F.sync()
    yr = M(x)
    assert np.linalg.norm(y.cpu().numpy() - yr) <= 1e-10 * np.linalg.norm(yr)
    # repeated applies reuse the prepared solve
    y2 = F.apply(torch.from_numpy(x).cuda())
    F.sync()
    assert np.array_equal(y.cpu().numpy(), y2.cpu().numpy())


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_bicgstab_iterations_match_oracle(D, alg):
    w = make_workload("convdiff32")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg)
    S = D.Solver(D.DeviceCSC.from_host(w.A))
    b = torch.from_numpy(w.b).cuda()
    x, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg)
    xo, its, rr, st = O.bicgstab(w.A.to_scipy(), w.b, O.Preconditioner(o.W_csc(), o.V_csc()))
    assert info.converged == 1 and st == "ok"
    assert abs(info.iterations - its) <= 1
    assert np.allclose(x.cpu().numpy(), 1.0, atol=1e-5)
    x0, info0 = S.bicgstab(b, None, tol=1e-8, maxit=1000)
    assert info0.converged and info.iterations < info0.iterations


@pytest.mark.parametrize("name", ["helmholtz40", "convdiff32"])
def test_gmres_matches_oracle(D, name):
    """GMRES(50) to 1e-6 with the preconditioner (the solver of Sec. 5 for
    the complex problem): iteration count within 2 of the oracle's GMRES."""
    w = make_workload(name)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    S = D.Solver(D.DeviceCSC.from_host(w.A))
    b = torch.from_numpy(w.b).cuda()
    x, info = S.gmres(b, F, tol=1e-6, restart=50, maxit=2000)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    xo, its, rr, st = O.gmres(w.A.to_scipy(), w.b, O.Preconditioner(o.W_csc(), o.V_csc()), restart=50, tol=1e-6)
    assert info.converged == 1 and st == "ok"
    assert abs(info.iterations - its) <= 2, (info.iterations, its)
    r = w.b - w.A.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) <= 1.01e-6 * np.linalg.norm(w.b)
    # a short restart length forces several cycles
    x5, info5 = S.gmres(b, F, tol=1e-6, restart=5, maxit=5000)
    xo5, its5, _, st5 = O.gmres(w.A.to_scipy(), w.b, O.Preconditioner(o.W_csc(), o.V_csc()), restart=5, tol=1e-6,
                                maxit=5000)
    assert info5.converged == (st5 == "ok")
    if st5 == "ok":
        assert abs(info5.iterations - its5) <= max(3, its5 // 20), (info5.iterations, its5)
    x0, info0 = S.gmres(b, None, tol=1e-6, restart=50, maxit=4000)
    assert info.iterations < info0.iterations
