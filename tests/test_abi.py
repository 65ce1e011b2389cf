"""The C ABI library: it builds, loads, exports every symbol include/*.h
declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(diaf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1208_3573_gb300 import build
    build.build()
    from paper_1208_3573_gb300 import diaf
    return diaf.lib()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("diaf_factor", "diaf_apply", "diaf_get_factors", "diaf_free", "diaf_status_string", "diaf_bicgstab"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(7):
        assert lib.diaf_status_string(s)
    assert lib.diaf_status_string(99) == b"unknown status"


def test_host_side_argument_errors(lib):
    from paper_1208_3573_gb300 import diaf
    out = ctypes.c_void_p()
    a = diaf.CSC_t(4, 0, None, None, None, 0)
    pw = diaf.Pattern_t(4, 0, None, None)
    vs = diaf.VSpec_t(1, None, None, 0.0)
    # NULL out pointer, bad alg, bad dtype, size mismatch, NULL arrays: all rejected before any CUDA call
    assert lib.diaf_factor(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), 2, 0, None, None) == 1
    assert lib.diaf_factor(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), 7, 0, None, ctypes.byref(out)) == 1
    a_bad = diaf.CSC_t(4, 0, None, None, None, 9)
    assert lib.diaf_factor(ctypes.byref(a_bad), ctypes.byref(pw), ctypes.byref(vs), 2, 0, None,
                           ctypes.byref(out)) == 1
    pw_bad = diaf.Pattern_t(5, 0, None, None)
    assert lib.diaf_factor(ctypes.byref(a), ctypes.byref(pw_bad), ctypes.byref(vs), 2, 0, None,
                           ctypes.byref(out)) == 1
    assert lib.diaf_factor(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs), 2, 0, None, ctypes.byref(out)) == 1
    assert b"NULL" in lib.diaf_last_error()
    vs_bad = diaf.VSpec_t(0, None, None, 0.0)  # fixed rule without a pattern
    assert lib.diaf_factor(ctypes.byref(a), ctypes.byref(pw), ctypes.byref(vs_bad), 2, 0, None,
                           ctypes.byref(out)) == 1
    assert out.value is None


def test_product_path_has_no_oracle_dependency():
    """The CUDA path never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1208_3573_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            for pat in ("import oracle", "from oracle", "libdiaf_oracle", "diaf_oracle"):
                assert pat not in src, (f, pat)
