"""Mixed-precision form (FP32 factorisations + one FP64 refinement step)
against the FP64 oracle: I_j bit-exact, per-column residual within 1e-4
relative, w_j / v_j within 1e-6 up to phase where unique; the columns the
FP32 path could not decide (flag FP64_FALLBACK) are computed by the FP64
kernel and must meet the same bar."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from tests._parity import assert_parity, compare, host_factors
from tests._problems import random_sparse
from tests.test_gpu_parity import run_gpu
from workloads import diagonal_pattern, make_workload, pattern_of, upper_budget

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL_RES, VEC_TOL = 1e-4, 1e-6


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name", ["convdiff32", "convdiff48_A2", "helmholtz40", "lognormal16", "powerlaw6k"])
def test_mixed_parity_workloads(D, name, alg):
    w = make_workload(name)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, prec="mixed32", tie_tol=w.tie_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    rep = compare(g, o, w.A, w.PW, alg, rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10)
    assert_parity(rep)
    fb = F.fallbacks()
    assert sum(fb) == int(np.count_nonzero(g["flags"] & 64))


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("cplx", [False, True])
def test_mixed_parity_random_fixed_and_rules(D, alg, cplx):
    A = random_sparse(300, 0.015, 17, cplx)
    PW = pattern_of(A)
    for vrule, budget, Vf in ((O.RULE_UPPER, upper_budget(A), None), (O.RULE_LOWER, None, None),
                              (O.RULE_ALL, np.full(A.n, 4, np.int32), None),
                              (O.RULE_FIXED, None, diagonal_pattern(A.n)),
                              (O.RULE_FIXED, None, pattern_of(sp.triu(A.to_scipy())))):
        F = run_gpu(D, A, PW, vrule, budget, Vf, alg=alg, prec="mixed32")
        g = host_factors(F)
        o = O.factor(A, PW, vrule, budget, Vf, alg=alg)
        assert_parity(compare(g, o, A, PW, alg, rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10))


def test_mixed_bicgstab_matches_fp64(D):
    w = make_workload("convdiff32")
    S = D.Solver(D.DeviceCSC.from_host(w.A))
    b = torch.from_numpy(w.b).cuda()
    its = {}
    for prec in ("fp64", "mixed32"):
        F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec=prec)
        x, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
        assert info.converged
        its[prec] = info.iterations
    assert abs(its["fp64"] - its["mixed32"]) <= 1


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_mixed_parity_full_size_convdiff256(D, alg):
    """The benchmark's workload (65,536 columns) in mixed precision, every column."""
    w = make_workload("convdiff256_A2")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, prec="mixed32", tie_tol=w.tie_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    rep = compare(g, o, w.A, w.PW, alg, rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10)
    assert_parity(rep)
    # the FP32 path decides almost every column of this workload itself
    assert sum(F.fallbacks()) <= 0.01 * w.n
    # the largest residual difference, over columns whose residual is above the rounding floor
    resg, reso = g["res"], o.res
    big = reso > 1e-10 * np.abs(w.A.vals).max()
    print(alg, "max rel res diff", float(np.max(np.abs(resg[big] - reso[big]) / reso[big])), "cols", int(big.sum()))


def test_mixed_parity_full_size_powerlaw_sampled(D):
    """n = 200,000, all three buckets in mixed precision (the large tiles in the
    mixed CTA kernel): every column of the largest bucket up to 1,500 plus a
    seeded sample of the others."""
    w = make_workload("powerlaw200k")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec="mixed32", tie_tol=w.tie_tol)
    g = host_factors(F)
    k = w.PW.counts()
    nnz = np.diff(w.A.colptr)
    E = np.bincount(np.repeat(np.arange(w.n), k), weights=nnz[w.PW.rowidx], minlength=w.n)
    big = np.nonzero((k > 32) | (E > 200))[0]
    rng = np.random.default_rng(5)
    cols = np.unique(np.concatenate([big[:1500], rng.choice(w.n, 1500, replace=False)])).astype(np.int32)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol, cols=cols)
    rep = compare(g, o, w.A, w.PW, "S", rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10, cols=cols)
    assert_parity(rep)
    fb = F.fallbacks()
    assert fb[2] < F.info.bucket_cols[2]  # the mixed CTA kernel finished part of the large bucket
    print("fallbacks per bucket", fb, "of", list(F.info.bucket_cols))


def test_mixed_close_pairs_powerlaw(D):
    """Columns whose two smallest singular values of A-hat are close (sigma^2
    gap at most 1e-5 ||T||_F^2, a superset of the kernels' close-pair test
    against sigma_max^2): the large-tile kernel resolves such a pair by FP64
    corrections of both vectors and a 2 x 2 Rayleigh-Ritz step instead of
    handing the column to the FP64 kernel.  Every such column of n = 200,000
    must be at parity (unique vectors within 1e-6, DEGENERATE from the FP64
    Ritz values), and few of the large bucket's columns may go to FP64."""
    w = make_workload("powerlaw200k")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec="mixed32", tie_tol=w.tie_tol)
    g = host_factors(F)
    o_all = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    colnorm2 = np.bincount(np.repeat(np.arange(w.n), np.diff(w.A.colptr)), weights=w.A.vals ** 2, minlength=w.n)
    k = w.PW.counts()
    tf2 = np.bincount(np.repeat(np.arange(w.n), k), weights=colnorm2[w.PW.rowidx], minlength=w.n)
    s0, s1 = o_all.sig[:, 0], o_all.sig[:, 1]
    close = np.nonzero((k > 1) & (s1 ** 2 - s0 ** 2 <= 1e-5 * tf2))[0].astype(np.int32)
    assert close.size > 100
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol, cols=close)
    rep = compare(g, o, w.A, w.PW, "S", rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10, cols=close)
    assert_parity(rep)
    fb = F.fallbacks()
    kept = int(np.count_nonzero((g["flags"][close] & 64) == 0))
    print("close columns", close.size, "kept in mixed precision", kept, "fallbacks per bucket", fb)
    assert fb[2] < 100


@pytest.mark.parametrize("alg", ["S", "Q"])
def test_mixed_parity_full_size_lognormal64(D, alg):
    """262,144 columns with k = 25 tiles: every I_j of the mixed form must be the
    FP64 choice (the key-error bound decides which columns the FP64 kernel takes)."""
    w = make_workload("lognormal64")
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, prec="mixed32", tie_tol=w.tie_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    assert_parity(compare(g, o, w.A, w.PW, alg, rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10))


@pytest.mark.parametrize("small", [1, 2])
@pytest.mark.parametrize("name", ["convdiff32", "convdiff48_A2", "powerlaw6k", "lognormal16", "convdiff256_A2"])
def test_small_tile_kernels_at_parity(D, name, small):
    """Size bucket 0 of real DIAF-S in mixed precision runs one thread per
    column (small_tiles 1, the default; columns it cannot finish in FP32 go on
    to the warp kernel) or one warp per column (2): both at parity with the
    oracle on every column."""
    w = make_workload(name)
    dA = D.DeviceCSC.from_host(w.A)
    dP = D.DeviceCSC.from_host(w.PW)
    dB = torch.from_numpy(w.budget).cuda()
    F = D.factor(dA, dP, w.vrule, dB, alg="S", prec="mixed32", tie_tol=w.tie_tol, tuning={"small_tiles": small})
    torch.cuda.synchronize()
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    assert_parity(compare(g, o, w.A, w.PW, "S", rtol_res=RTOL_RES, vec_tol=VEC_TOL, mixed=True, floor_rel=1e-10))
