"""The apply (y = W V^-1 x) on the V structures other than the upper rule's:
a lower-triangular V (its solve runs in increasing row order), a fixed upper
pattern, and the two errors the apply's preparation reports -- V neither
upper nor lower triangular, and a zero or missing diagonal entry -- against
the oracle's preconditioner.  The level schedule of V is computed on the
host from V's columns, so these cases exercise both solve orders and the
structure checks of that pass.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from tests._problems import pattern_from_sets, random_sparse
from workloads import lower_budget, make_workload, pattern_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


def factor(D, A, PW, vrule, budget=None, Vfixed=None, alg="S", prec="fp64"):
    dA = D.DeviceCSC.from_host(A)
    dP = D.DeviceCSC.from_host(PW)
    dB = None if budget is None else torch.from_numpy(np.ascontiguousarray(budget, np.int32)).cuda()
    dV = None if Vfixed is None else D.DeviceCSC.from_host(Vfixed)
    F = D.factor(dA, dP, vrule, dB, dV, alg=alg, prec=prec)
    torch.cuda.synchronize()
    return F


def vector(A, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n)
    if A.is_complex:
        x = x + 1j * rng.standard_normal(A.n)
    return x


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("name", ["convdiff32", "helmholtz40"])
@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
def test_apply_lower_rule_and_fixed_upper(D, alg, name, prec):
    w = make_workload(name)
    A, PW = w.A, w.PW
    # (the lower rule without a budget takes every admissible row: its V^-1 x grows to ~1e36 on
    # these operators, where rounding differences decide the digits -- not a usable preconditioner)
    for vrule, budget, Vf in ((O.RULE_LOWER, lower_budget(A), None),
                              (O.RULE_FIXED, None, pattern_of(sp.triu(A.to_scipy())))):
        F = factor(D, A, PW, vrule, budget, Vf, alg=alg, prec=prec)
        o = O.factor(A, PW, vrule, budget, Vf, alg=alg)
        x = vector(A, 1)
        y = F.apply(torch.from_numpy(x).cuda())
        F.sync()
        yr = O.Preconditioner(o.W_csc(), o.V_csc())(x)
        # the mixed form's W and V agree with the FP64 ones to ~1e-13 (relative); V^-1 can amplify that
        tol = 1e-10 if prec == "fp64" else 1e-8
        assert np.linalg.norm(y.cpu().numpy() - yr) <= tol * np.linalg.norm(yr), (vrule, alg, prec)


def test_apply_rejects_a_v_that_is_not_triangular(D):
    A = random_sparse(64, 0.08, 5)
    PW = pattern_of(A)
    n = A.n
    tri = pattern_from_sets(n, [[r for r in (j - 1, j, j + 1) if 0 <= r < n] for j in range(n)])
    F = factor(D, A, PW, O.RULE_FIXED, None, tri)
    with pytest.raises(D.DiafError) as e:
        F.apply(torch.from_numpy(vector(A, 2)).cuda())
    assert e.value.status == D.DIAF_EINVAL and "triangular" in str(e.value)


@pytest.mark.parametrize("upper", [True, False])
def test_apply_rejects_a_missing_diagonal_entry(D, upper):
    A = random_sparse(64, 0.08, 6)
    PW = pattern_of(A)
    n = A.n
    sets = [[j] for j in range(n)]
    sets[10] = [9] if upper else [11]  # column 10 without its diagonal, V still triangular
    F = factor(D, A, PW, O.RULE_FIXED, None, pattern_from_sets(n, sets))
    with pytest.raises(D.DiafError) as e:
        F.apply(torch.from_numpy(vector(A, 3)).cuda())
    assert e.value.status == D.DIAF_EINVAL and "diagonal" in str(e.value)
