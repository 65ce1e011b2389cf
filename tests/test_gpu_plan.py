"""Launch tuning, the CUDA-graph plan and the autotuner: each must produce the
same W, V as the method (checked against the oracle, or bit-for-bit against
the untuned call where the kernels are the same)."""
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


def _dev(D, w):
    return D.DeviceCSC.from_host(w.A), D.DeviceCSC.from_host(w.PW), torch.from_numpy(w.budget).cuda()


@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("tuning", [{"m_edge0": 16, "m_edge1": 48}, {"m_edge0": 24, "warps_per_block": [2, 1]},
                                    {"m_edge1": 32, "warps_per_block": [8, 4]}])
def test_tuned_buckets_match_oracle(D, prec, tuning):
    w = make_workload("powerlaw6k")
    A, PW, bud = _dev(D, w)
    F = D.factor(A, PW, w.vrule, bud, alg="S", prec=prec, tie_tol=w.tie_tol, tuning=tuning)
    torch.cuda.synchronize()
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    kw = dict(rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10) if prec == "mixed32" else {}
    assert_parity(compare(g, o, w.A, w.PW, "S", **kw))


@pytest.mark.parametrize("alg", ["S", "Q"])
@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("name,tuned", [("convdiff48_A2", False), ("powerlaw6k", False), ("powerlaw6k", True)])
def test_plan_replay_matches_factor_and_tracks_new_values(D, name, tuned, alg, prec):
    """One graph over the size buckets (with the default edges the power-law
    operator fills all three), with the default or the autotuner's launch
    tuning, replayed on new values."""
    w = make_workload(name)
    A, PW, bud = _dev(D, w)
    tuning = None
    if tuned:
        tuning, _ = D.autotune(A, PW, w.vrule, bud, alg=alg, prec=prec, tie_tol=w.tie_tol)
    ref = host_factors(D.factor(A, PW, w.vrule, bud, alg=alg, prec=prec, tie_tol=w.tie_tol, tuning=tuning))
    P = D.Plan(A, PW, w.vrule, bud, alg=alg, prec=prec, tie_tol=w.tie_tol, tuning=tuning)
    if name == "powerlaw6k" and not tuned:
        info = P.execute().info
        assert all(info.bucket_cols[b] > 0 for b in range(info.n_buckets))
    g = host_factors(P.execute())
    for key in ("Vcp", "Vri", "flags"):
        assert np.array_equal(g[key], ref[key])
    for key in ("Wv", "Vv", "res"):
        assert np.array_equal(g[key], ref[key])  # same kernels, same inputs
    # new values in the same buffer (a different operator on the same structure)
    rng = np.random.default_rng(5)
    newvals = w.A.vals * (1.0 + 0.3 * rng.standard_normal(w.A.nnz))
    A.vals.copy_(torch.from_numpy(newvals))
    g2 = host_factors(P.execute())
    torch.cuda.synchronize()
    A2 = type(w.A)(w.A.n, w.A.colptr, w.A.rowidx, newvals)
    o = O.factor(A2, w.PW, w.vrule, w.budget, alg=alg, tie_tol=w.tie_tol)
    kw = dict(rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10) if prec == "mixed32" else {}
    assert_parity(compare(g2, o, A2, w.PW, alg, **kw))


def test_autotune_returns_a_working_tuning(D):
    w = make_workload("powerlaw6k")
    A, PW, bud = _dev(D, w)
    tuning, ms = D.autotune(A, PW, w.vrule, bud, alg="S", prec="mixed32", tie_tol=w.tie_tol)
    assert ms > 0
    assert 0 <= tuning["m_edge0"] <= 32 and 0 <= tuning["m_edge1"] <= 64
    F = D.factor(A, PW, w.vrule, bud, alg="S", prec="mixed32", tie_tol=w.tie_tol, tuning=tuning)
    g = host_factors(F)
    o = O.factor(w.A, w.PW, w.vrule, w.budget, alg="S", tie_tol=w.tie_tol)
    assert_parity(compare(g, o, w.A, w.PW, "S", rtol_res=1e-4, vec_tol=1e-6, mixed=True, floor_rel=1e-10))
