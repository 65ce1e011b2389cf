"""diaf_apply_static -- the preconditioner apply for callers that cannot
allocate device memory when they apply it: code held to a device-memory
budget fixed at start-up, or a host framework whose allocator owns all device
memory and forbids allocations by the libraries it calls.  Its scratch is a
fixed array inside the library instead of buffers of the factor handle.

Checked through the C ABI against diaf_apply on the same factors and against
the oracle's W V^-1 (a sparse LU of the oracle's V), on two calls in a row
with different inputs (the second call reuses the array the first one left
behind), for upper and lower triangular V, real and complex."""
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


@pytest.mark.parametrize("name,lower", [("convdiff32", False), ("helmholtz40", False), ("convdiff32", True)])
def test_apply_static_matches_apply(D, name, lower):
    w = make_workload(name)
    rule, budget = (O.RULE_LOWER, lower_budget(w.A)) if lower else (w.vrule, w.budget)
    F = D.factor(D.DeviceCSC.from_host(w.A), D.DeviceCSC.from_host(w.PW), rule,
                 torch.from_numpy(budget).cuda(), alg="S", tie_tol=w.tie_tol)
    o = O.factor(w.A, w.PW, rule, budget, alg="S", tie_tol=w.tie_tol)
    M = O.Preconditioner(o.W_csc(), o.V_csc())
    rng = np.random.default_rng(7)
    dt = torch.complex128 if w.A.is_complex else torch.float64

    def vec():
        return rng.standard_normal(w.n) + (1j * rng.standard_normal(w.n) if w.A.is_complex else 0)

    y = torch.empty(w.n, dtype=dt, device="cuda")
    with pytest.raises(D.DiafError):  # no row-oriented copies yet: it will not build (allocate) them
        F.apply_static(torch.from_numpy(vec()).to("cuda", dt), y)
    for _ in range(2):
        xh = vec()
        x = torch.from_numpy(xh).to("cuda", dt)
        ref = F.apply(x)
        out = torch.full_like(ref, float("nan"))
        F.apply_static(x, out)
        F.sync()
        r = ref.cpu().numpy(); got = out.cpu().numpy(); yo = M(xh)
        assert np.linalg.norm(got - r) <= 1e-10 * np.linalg.norm(r)
        assert np.linalg.norm(got - yo) <= 1e-10 * np.linalg.norm(yo)


def test_apply_static_rejects_oversize(D):
    from workloads import CSC, Pattern
    n = (1 << 18) + 1  # one row beyond the limit: diagonal matrix
    A = CSC(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    P = Pattern(n, A.colptr, A.rowidx)
    F = D.factor(D.DeviceCSC.from_host(A), D.DeviceCSC.from_host(P), 1, None, alg="S")
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    F.apply(x)
    with pytest.raises(D.DiafError) as e:
        F.apply_static(x, torch.empty_like(x))
    assert e.value.status == D.DIAF_EINVAL and "limit" in str(e.value)
