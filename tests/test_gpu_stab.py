"""Stabilised DIAF-Q (Sec. 3.2) on the GPU against the oracle: every
workload with the paper's trigger |v_jj| < 1e-2 and with the trigger always
on (stab_tol = 2), FP64 (warp and CTA kernels) and mixed precision (columns
at the trigger go to the FP64 kernel).  Same bar as the plain method; the
STABILISED flag must match column by column."""
import numpy as np
import pytest

import oracle as O
from tests._parity import assert_parity, compare, host_factors
from tests.test_gpu_parity import run_gpu
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


@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("stab_tol", [1e-2, 2.0])
@pytest.mark.parametrize("name", ["convdiff48_A2", "helmholtz40", "lognormal16", "powerlaw6k"])
def test_stabilised_parity(D, name, stab_tol, prec):
    w = make_workload(name)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="Q", prec=prec, tie_tol=w.tie_tol, stab_tol=stab_tol)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="Q", tie_tol=w.tie_tol, stab_tol=stab_tol)
    kw = dict(rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10) if prec == "mixed32" else {}
    assert_parity(compare(g, o, w.A, w.PW, "Q", **kw))
    n_stab = int(np.sum((o.flags & O.F_STABILISED) != 0))
    if stab_tol > 1:
        assert n_stab >= int(np.sum(np.diff(o.voff) > 1)) > 0  # every column with l_j > 1
    # stabilised columns carry v_jj = r / sqrt(r^2 + 1) on the GPU too
    st = np.nonzero(g["flags"] & O.F_STABILISED)[0]
    for j in st[:200]:
        lo, hi = g["Vcp"][j], g["Vcp"][j + 1]
        vjj = g["Vv"][lo:hi][g["Vri"][lo:hi] == j][0]
        assert abs(vjj - 2 / np.sqrt(5)) < 1e-12
