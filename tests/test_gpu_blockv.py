"""Block-diagonal V (DIAF_RULE_BLOCK; the V structure of Sec. 5's
experiments) on the GPU: factorisation against the oracle (I_j bit-exact,
residuals, vectors), the block-LU apply against the oracle's sparse LU of V,
BiCGSTAB iteration counts, and the input errors."""
import numpy as np
import pytest

import oracle as O
from tests._parity import assert_parity, compare, host_factors
from workloads import make_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


def _run(D, w, blocks, budget, alg, prec):
    A = D.DeviceCSC.from_host(w.A)
    PW = D.DeviceCSC.from_host(w.PW)
    b = torch.from_numpy(np.ascontiguousarray(budget, np.int32)).cuda()
    blk = torch.from_numpy(np.ascontiguousarray(blocks, np.int32)).cuda()
    F = D.factor(A, PW, D.RULE_BLOCK, b, alg=alg, prec=prec, tie_tol=w.tie_tol, blocks=blk)
    torch.cuda.synchronize()
    return F


@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name,bsize,kv", [("convdiff48_A2", 48, 6), ("lognormal16", 64, 8), ("helmholtz40", 20, 5),
                                           ("powerlaw6k", 50, 4)])
def test_block_parity(D, name, bsize, kv, alg, prec):
    w = make_workload(name)
    blocks = np.arange(w.n) // bsize
    budget = np.full(w.n, kv, np.int32)
    F = _run(D, w, blocks, budget, alg, prec)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, O.RULE_BLOCK, budget, None, alg=alg, tie_tol=w.tie_tol, blocks=blocks)
    kw = dict(rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10) if prec == "mixed32" else {}
    assert_parity(compare(g, o, w.A, w.PW, alg, **kw))


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name,bsize", [("convdiff32", 32), ("helmholtz40", 40), ("lognormal16", 64)])
def test_block_apply_matches_oracle(D, name, bsize, alg):
    w = make_workload(name)
    blocks = np.arange(w.n) // bsize
    budget = np.full(w.n, 6, np.int32)
    F = _run(D, w, blocks, budget, alg, "fp64")
    o = O.factor(w.A, w.PW, O.RULE_BLOCK, budget, None, alg=alg, tie_tol=w.tie_tol, blocks=blocks)
    M = O.Preconditioner(o.W_csc(), o.V_csc())
    rng = np.random.default_rng(1)
    x = rng.standard_normal(w.n) + (1j * rng.standard_normal(w.n) if w.A.is_complex else 0)
    y = F.apply(torch.from_numpy(x).cuda())
    F.sync()
    yr = M(x)
    # W and V agree with the oracle's to ~1e-10; V^-1 amplifies that by its
    # condition number, the largest over the diagonal blocks
    Vd = o.V_csc().tocsc()
    kappa = max(np.linalg.cond(Vd[b0:b0 + bsize, b0:b0 + bsize].toarray()) for b0 in range(0, w.n, bsize))
    assert np.linalg.norm(y.cpu().numpy() - yr) <= 1e-10 * max(10.0, kappa) * np.linalg.norm(yr)


def test_block_bicgstab_matches_oracle(D):
    w = make_workload("convdiff32")
    blocks = np.arange(w.n) // 32
    budget = np.full(w.n, 8, np.int32)
    F = _run(D, w, blocks, budget, "S", "mixed32")
    S = D.Solver(D.DeviceCSC.from_host(w.A))
    b = torch.from_numpy(w.b).cuda()
    x, info = S.bicgstab(b, F, tol=1e-8, maxit=1000)
    o = O.factor(w.A, w.PW, O.RULE_BLOCK, budget, None, alg="S", tie_tol=w.tie_tol, blocks=blocks)
    xo, its, rr, st = O.bicgstab(w.A.to_scipy(), w.b, O.Preconditioner(o.W_csc(), o.V_csc()))
    assert info.converged == 1 and st == "ok"
    assert abs(info.iterations - its) <= 1
    assert np.allclose(x.cpu().numpy(), 1.0, atol=1e-5)


def test_block_errors(D):
    w = make_workload("convdiff32")
    budget = np.full(w.n, 4, np.int32)
    F = _run(D, w, np.arange(w.n) // 80, budget, "S", "fp64")  # blocks of 80 rows
    x = torch.ones(w.n, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DiafError) as e:
        F.apply(x)
    assert e.value.status == D.DIAF_EUNSUPPORTED
    dec = (np.arange(w.n) // 32)[::-1].copy()  # decreasing block ids
    F = _run(D, w, dec, budget, "S", "fp64")
    with pytest.raises(D.DiafError) as e:
        F.apply(x)
    assert e.value.status == D.DIAF_EINVAL
    F = _run(D, w, np.arange(w.n) // 32, budget, "S", "fp64")
    F.apply(x)
    y = torch.empty_like(x)
    with pytest.raises(D.DiafError) as e:
        F.apply_static(x, y)
    assert e.value.status == D.DIAF_EUNSUPPORTED
