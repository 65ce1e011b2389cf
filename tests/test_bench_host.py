"""Host logic of bench.py that needs no GPU: the clock sampler's summary of
nvidia-smi lines (reasons, medians, the fallback to the sample taken before a
short timed region) and the algorithmic flop count's closed form."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.00, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_during_region():
    c = bench.ClockSampler(0)
    c.first = _line(2070, 2070) + "\n"
    c.out = "\n".join([_line(2070, 2070), _line(2055, 2070, cap="Active"), _line(2070, 2070)]) + "\n"
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and "note" not in s


def test_clock_summary_flags_throttling():
    c = bench.ClockSampler(0)
    c.first = ""
    c.out = _line(1500, 2070, hwt="Active") + "\n"
    s = c.summary()
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_short_region_falls_back_to_the_first_sample():
    c = bench.ClockSampler(0)
    c.first = _line(2070, 2070) + "\n"
    c.out = ""
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] == 2070.0 and "note" in s


def test_clock_summary_without_sampler():
    c = bench.ClockSampler(0)
    c.first, c.out = "", ""
    assert c.summary()["reasons"] == ["unsampled"]


def test_algorithmic_flops_closed_form():
    # one column, k = 2, m = 3, l = 1, real DIAF-S with 5 Jacobi sweeps: QR of T
    # 2k^2(m - k/3), leverage m k^2, QR of A-hat 2k^2(max(m - l, k) - k/3), Jacobi
    # 5 sweeps x k(k-1)/2 pairs x 14 k, FP64 correction 4 m k, v and residual 2 m k
    m, k, l = np.array([3]), np.array([2]), np.array([1])
    f64 = 4 * 3 * 2 + 2 * 3 * 2
    want = 2 * 4 * (3 - 2 / 3) + 3 * 4 + 2 * 4 * (max(3 - 1, 2) - 2 / 3) + 5 * 1 * 14 * 2 + f64
    got, got64 = bench.algorithmic_flops(m, k, l, "S", False, sweeps=5)
    assert abs(got - want) < 1e-9 * want and abs(got64 - f64) < 1e-9 * f64
    got_c, got64_c = bench.algorithmic_flops(m, k, l, "S", True, sweeps=5)
    assert abs(got_c - 4 * want) < 1e-9 * want and abs(got64_c - 4 * f64) < 1e-9 * f64


def test_gathered_bytes():
    from workloads import CSC, Pattern
    # 3 x 3: column nnz 2, 1, 3; W pattern uses column 0 twice and column 2 once
    A = CSC(3, np.array([0, 2, 3, 6], np.int32), np.array([0, 1, 1, 0, 1, 2], np.int32), np.ones(6))
    P = Pattern(3, np.array([0, 1, 2, 3], np.int32), np.array([0, 0, 2], np.int32))

    class Wl:
        pass
    w = Wl(); w.A, w.PW = A, P
    assert bench.gathered_bytes(w) == (2 + 2 + 3) * 12.0


def test_dominant_kernel_names_the_bucket_kernel():
    assert bench.dominant_kernel(0, "mixed32", "S", False).startswith("column_thread_kernel")
    assert bench.dominant_kernel(1, "mixed32", "S", False) == "column_mixed_kernel"
    assert bench.dominant_kernel(2, "mixed32", "S", False) == "column_cta_mixed_kernel"
    assert bench.dominant_kernel(2, "mixed32", "Q", False).startswith("column_cta_kernel")
    assert bench.dominant_kernel(0, "mixed32", "S", True) == "column_mixed_kernel"
    assert bench.dominant_kernel(1, "fp64", "S", False) == "column_warp_kernel"
    assert bench.dominant_kernel(2, "fp64", "Q", True) == "column_cta_kernel"
