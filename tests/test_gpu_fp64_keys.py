"""The mixed form's in-kernel FP64 leverage keys (taken by a column whose FP32
key decision is within the FP32 error bound of its threshold) on every rule
column: a separate build with a huge bound sends all of them through that
path, real and complex, both algorithms, warp and CTA kernels, and the results
must stay at parity with the oracle.  Runs in a child process, which loads that
build instead of the library of the other tests."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64_key_path_on_every_column():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = subprocess.run([sys.executable, "-m", "tests._fp64_keys_check"], cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
