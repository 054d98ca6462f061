"""The roofline arithmetic of bench.py on made-up timings (no GPU): the
headline fraction is the oracle's work per substep x substeps / time over
the peak of the kernel's precision, the kernel-counted one the executed
flops over the busiest pipe's peak, and the peaks are unit counts x clock."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _res(leg, substeps=1.0e9, calls=1, ms=100.0):
    return {leg: {"stats": {"substeps": substeps, "calls": calls}, "ms": ms}}


def test_peaks_from_unit_counts(bench):
    clk = {"sm_max_mhz": 2070.0}
    r = bench.roofline(_res("mixed"), clk, 1000, "mixed", None)
    assert r["kernel_counted"]["peak"] == pytest.approx(152 * 4 * 2070e6 / 1e12)          # FP64
    assert r["kernel_counted"]["other"]["peak"] == pytest.approx(152 * 256 * 2070e6 / 1e12)  # FP32


def test_algorithmic_headline(bench):
    clk = {"sm_max_mhz": 2000.0}
    alg = {"flops_per_substep": 4000.0, "transcendentals_per_substep": 60.0}
    r = bench.roofline(_res("mixed", substeps=2.0e9, calls=2, ms=50.0), clk, 1000, "mixed", alg)
    ach = 4000.0 * 1.0e9 / 0.05 / 1e12                      # per launch: 1e9 substeps in 50 ms
    assert r["achieved"] == pytest.approx(ach)
    assert r["peak"] == pytest.approx(152 * 256 * 2000e6 / 1e12) and r["pipe"] == "fp32"
    assert r["frac"] == pytest.approx(ach / r["peak"])
    r64 = bench.roofline(_res("fp64", substeps=1.0e9, ms=1000.0), clk, 1000, "fp64", alg)
    assert r64["peak"] == pytest.approx(152 * 4 * 2000e6 / 1e12) and r64["pipe"] == "fp64"
    assert r64["frac"] == pytest.approx(4000.0 * 1.0e9 / 1.0 / 1e12 / r64["peak"])


def test_kernel_counted_picks_the_busier_pipe(bench):
    clk = {"sm_max_mhz": 2070.0}
    r = bench.roofline(_res("mixed", substeps=1.0e9, ms=100.0), clk, 1000, "mixed", None)
    w = bench.WORK_PER_SUBSTEP["mixed"]
    a64 = w["fp64_flops"] * 1.0e9 / 0.1 / 1e12
    a32 = w["fp32_flops"] * 1.0e9 / 0.1 / 1e12
    kc = r["kernel_counted"]
    p64 = 152 * 4 * 2070e6 / 1e12
    p32 = 152 * 256 * 2070e6 / 1e12
    assert kc["pipe"] == ("fp64" if a64 / p64 >= a32 / p32 else "fp32")
    assert kc["achieved"] == pytest.approx(a64 if kc["pipe"] == "fp64" else a32)
    # without the oracle's count the headline falls back to the kernel-counted figure
    assert r["frac"] == kc["frac"] and "kernel-counted" in r["work"]
    assert r["traffic"] == pytest.approx(bench.DRAM_BYTES_PER_CELL["mixed"] * 1000)
