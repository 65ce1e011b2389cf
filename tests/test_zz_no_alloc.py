"""diaf_apply_static -- the preconditioner apply for callers that cannot
allocate device memory when they apply it (fixed memory budgets, solver loops
recorded into CUDA graphs, host frameworks that own all device memory).  Its
scratch is a fixed array inside the library instead of buffers of the factor
handle.  Checked through the C ABI against diaf_apply on the same factors,
on two calls in a row with different inputs (the second call reuses the
array the first one left behind)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("name", ["convdiff32", "helmholtz40"])
def test_apply_static_matches_apply(D, name):
    w = make_workload(name)
    F = D.factor(D.DeviceCSC.from_host(w.A), D.DeviceCSC.from_host(w.PW), w.vrule,
                 torch.from_numpy(w.budget).cuda(), alg="S")
    rng = np.random.default_rng(7)
    dt = torch.complex128 if w.A.is_complex else torch.float64

    def vec():
        x = rng.standard_normal(w.n) + (1j * rng.standard_normal(w.n) if w.A.is_complex else 0)
        return torch.from_numpy(x).to("cuda", dt)

    y = torch.empty(w.n, dtype=dt, device="cuda")
    with pytest.raises(D.DiafError):  # no row-oriented copies yet: it will not build (allocate) them
        F.apply_static(vec(), y)
    for _ in range(2):
        x = vec()
        ref = F.apply(x)
        out = torch.full_like(ref, float("nan"))
        F.apply_static(x, out)
        F.sync()
        r = ref.cpu().numpy(); o = out.cpu().numpy()
        assert np.linalg.norm(o - r) <= 1e-10 * np.linalg.norm(r)


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
