"""Failure paths, none of which faults, traps or hangs the GPU.

  * a NaN in A: the columns whose tile holds it are flagged NONFINITE, every
    other column is unchanged (bit for bit against a run on the clean A), the
    call itself succeeds;
  * a device-memory cap (diaf_set_device_memory_limit) below what the setup or
    the first apply needs: DIAF_ENOMEM, nothing left allocated, and the same
    calls succeed once the cap is lifted;
  * a build of the library with the Jacobi sweep limit at 1 (run in a child
    process that loads that build): JACOBI_NOCONV is set and the results stay
    finite.

No kernel of the library waits on a flag or on another block (the
triangular solves are level-scheduled), so there is no bounded wait whose
timeout path a test would have to exercise."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests._parity import F_NONFIN, host_factors
from tests.test_gpu_parity import run_gpu
from workloads import CSC, make_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1208_3573_gb300 import build, diaf
    build.build()
    return diaf


@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("alg", ["S", "Q"])
def test_nan_in_A_flags_nonfinite(D, alg, prec):
    w = make_workload("convdiff32")
    c = 500
    p = int(np.searchsorted(w.A.rowidx[w.A.colptr[c]:w.A.colptr[c + 1]], c)) + int(w.A.colptr[c])
    vals = w.A.vals.copy()
    vals[p] = np.nan  # the diagonal entry of column c
    Abad = CSC(w.n, w.A.colptr, w.A.rowidx, vals)
    clean = host_factors(run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg=alg, prec=prec))
    F = run_gpu(D, Abad, w.PW, w.vrule, w.budget, alg=alg, prec=prec)
    F.sync()
    g = host_factors(F)
    hit = np.array([c in set(w.PW.col(j).tolist()) for j in range(w.n)])
    assert hit.sum() >= 3
    assert np.array_equal((g["flags"] & F_NONFIN) != 0, hit)
    ok = ~hit
    for key, cp in (("Wv", "Wcp"), ("Vv", "Vcp"), ("Vri", "Vcp")):
        for j in np.nonzero(ok)[0]:
            a, b = g[cp][j], g[cp][j + 1]
            assert np.array_equal(g[key][a:b], clean[key][a:b]), (key, j)
    assert np.array_equal(g["res"][ok], clean["res"][ok])
    assert np.array_equal(g["flags"][ok], clean["flags"][ok])


def test_device_memory_cap_gives_enomem(D):
    w = make_workload("convdiff256_A2")
    held = D.device_memory_in_use()
    try:
        D.set_device_memory_limit(held + (1 << 20))
        with pytest.raises(D.DiafError) as e:
            run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec="mixed32")
        assert e.value.status == D.DIAF_ENOMEM
        assert D.device_memory_in_use() == held  # what the failed call took is released
    finally:
        D.set_device_memory_limit(0)
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec="mixed32")
    x = torch.ones(w.n, dtype=torch.float64, device="cuda")
    try:  # the first apply allocates its row-oriented copies: capped too
        D.set_device_memory_limit(D.device_memory_in_use() + 4096)
        with pytest.raises(D.DiafError) as e:
            F.apply(x)
        assert e.value.status == D.DIAF_ENOMEM
    finally:
        D.set_device_memory_limit(0)
    y = F.apply(x)
    F.sync()
    assert torch.isfinite(y).all()
    F.close()
    assert D.device_memory_in_use() == held
    D.release_pool_memory()  # returns the pool's free memory; the next setup still works
    F = run_gpu(D, w.A, w.PW, w.vrule, w.budget, alg="S", prec="mixed32")
    F.sync()
    F.close()
    assert D.device_memory_in_use() == held
    with pytest.raises(D.DiafError):
        D.set_device_memory_limit(-1)


def test_sweep_cap_build():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = subprocess.run([sys.executable, "-m", "tests._failure_build_check"], cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
