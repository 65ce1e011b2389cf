"""The first apply's level schedule built from V's structure as the column
kernels hand it to the host during the numeric pass (the rows of each
finished column, then a per-column word; an upper V's columns are taken in
descending order).  Checked against the oracle's preconditioner W V^-1 and
against an apply whose schedule came from V's whole structure copied after
the pass: with the apply enqueued right after diaf_factor (the host walk then
waits on columns that are still being computed), for the upper and the lower
rule, on the kernels of every size bucket (four-lane, warp, 32-column, CTA),
FP64 and mixed forms; with two factorisations alive at once (the second goes
without the host copy); and with a factorisation freed before any apply
(which gives the copy back to the next one).
"""
import gc

import numpy as np
import pytest

import oracle as O
from workloads import lower_budget, make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


@pytest.fixture(autouse=True)
def _no_stale_factors():
    # factors left unreferenced by earlier tests are freed first, so that none
    # of them still holds the host copy of V's structure
    gc.collect()
    yield


def _inputs(D, w, rule):
    budget = lower_budget(w.A) if rule == O.RULE_LOWER else w.budget
    dA = D.DeviceCSC.from_host(w.A)
    dP = D.DeviceCSC.from_host(w.PW)
    dB = torch.from_numpy(np.ascontiguousarray(budget, np.int32)).cuda()
    return dA, dP, dB, budget


def _vector(w, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(w.n)
    if w.A.is_complex:
        x = x + 1j * rng.standard_normal(w.n)
    return x


def _reference(w, rule, budget, alg, x):
    o = O.factor(w.A, w.PW, rule, budget, alg=alg, tie_tol=w.tie_tol)
    return O.Preconditioner(o.W_csc(), o.V_csc())(x)


def _close(y, yr, tol):
    return np.linalg.norm(y - yr) <= tol * np.linalg.norm(yr)


@pytest.mark.parametrize("name,alg,prec,rule", [
    ("convdiff256_A2", "S", "mixed32", O.RULE_UPPER),   # four lanes per column (the headline kernel)
    ("convdiff256_A2", "Q", "mixed32", O.RULE_UPPER),   # mixed warp kernel
    ("convdiff48_A2", "S", "fp64", O.RULE_UPPER),       # FP64 warp kernel
    ("helmholtz40", "S", "mixed32", O.RULE_UPPER),      # complex mixed warp kernel
    ("lognormal16", "S", "mixed32", O.RULE_UPPER),      # 32-column warp kernel
    ("convdiff32", "S", "mixed32", O.RULE_LOWER),       # ascending walk
    ("convdiff32", "Q", "fp64", O.RULE_LOWER),
])
def test_streamed_schedule_matches_oracle(D, name, alg, prec, rule):
    w = make_workload(name)
    dA, dP, dB, budget = _inputs(D, w, rule)
    x = _vector(w, 3)
    dt = torch.complex128 if w.A.is_complex else torch.float64
    xd = torch.from_numpy(x).to("cuda", dt)
    torch.cuda.synchronize()
    s0, c0 = D.apply_prep_counts()
    F = D.factor(dA, dP, rule, dB, alg=alg, prec=prec, tie_tol=w.tie_tol)
    y = F.apply(xd)  # enqueued at once: the schedule is built while the numeric pass runs
    F.sync()
    s1, c1 = D.apply_prep_counts()
    assert (s1 - s0, c1 - c0) == (1, 0)
    y = y.cpu().numpy()
    tol = 1e-10 if prec == "fp64" else 1e-8
    assert _close(y, _reference(w, rule, budget, alg, x), tol)
    # a second apply on the same factors (level-ordered copies reused)
    y2 = F.apply(xd)
    F.sync()
    assert np.array_equal(y2.cpu().numpy(), y)
    F.close()


def test_two_factorisations_alive_at_once(D):
    w = make_workload("convdiff256_A2")
    dA, dP, dB, budget = _inputs(D, w, w.vrule)
    x = _vector(w, 5)
    xd = torch.from_numpy(x).cuda()
    s0, c0 = D.apply_prep_counts()
    F1 = D.factor(dA, dP, w.vrule, dB, alg="S", prec="mixed32", tie_tol=w.tie_tol)  # takes the host copy
    F2 = D.factor(dA, dP, w.vrule, dB, alg="S", prec="mixed32", tie_tol=w.tie_tol)  # goes without
    y2 = F2.apply(xd)
    y1 = F1.apply(xd)
    torch.cuda.synchronize()
    F1.sync()
    F2.sync()
    s1, c1 = D.apply_prep_counts()
    assert (s1 - s0, c1 - c0) == (1, 1)
    y1 = y1.cpu().numpy()
    y2 = y2.cpu().numpy()
    assert _close(y1, y2, 1e-13)
    assert _close(y1, _reference(w, w.vrule, budget, "S", x), 1e-8)
    F1.close()
    F2.close()


def test_free_before_apply_gives_the_copy_back(D):
    w = make_workload("convdiff48_A2")
    dA, dP, dB, budget = _inputs(D, w, w.vrule)
    x = _vector(w, 7)
    xd = torch.from_numpy(x).cuda()
    F0 = D.factor(dA, dP, w.vrule, dB, alg="S", prec="mixed32", tie_tol=w.tie_tol)
    F0.close()  # no apply: waits for its numeric pass, then releases the host copy
    s0, c0 = D.apply_prep_counts()
    F = D.factor(dA, dP, w.vrule, dB, alg="S", prec="mixed32", tie_tol=w.tie_tol)
    y = F.apply(xd)
    F.sync()
    s1, c1 = D.apply_prep_counts()
    assert (s1 - s0, c1 - c0) == (1, 0)
    assert _close(y.cpu().numpy(), _reference(w, w.vrule, budget, "S", x), 1e-8)
    F.close()


def test_streamed_structure_of_every_bucket(D):
    """The power-law operator's columns fill all three size buckets (four-lane
    and warp kernels, CTA kernels, FP64 hand-backs): every column reaches the
    host copy (the preparation counts as streamed), and the preparation then
    finds the zero diagonal entries this operator's upper V has (the oracle's
    V is exactly singular too), as it does from a copied structure."""
    w = make_workload("powerlaw6k")
    dA, dP, dB, budget = _inputs(D, w, w.vrule)
    xd = torch.ones(w.n, dtype=torch.float64, device="cuda")
    for prec in ("mixed32", "fp64"):
        torch.cuda.synchronize()
        s0, c0 = D.apply_prep_counts()
        F = D.factor(dA, dP, w.vrule, dB, alg="S", prec=prec, tie_tol=w.tie_tol)
        bc = [F.info.bucket_cols[b] for b in range(3)]
        assert sum(bc) == w.n and min(bc) > 0, bc
        with pytest.raises(D.DiafError) as e:
            F.apply(xd)
        assert e.value.status == D.DIAF_EINVAL and "diagonal" in str(e.value)
        s1, c1 = D.apply_prep_counts()
        assert (s1 - s0, c1 - c0) == (1, 0), prec
        F.close()
