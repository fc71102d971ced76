"""bench.py's host logic (no GPU): the clock record taken during the timed
region (median SM clock, throttle reasons seen as Active), the FP32 peak
derived from the unit counts, and the whole-job throughput."""

import pytest

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s


def test_clock_summary_takes_the_median_and_every_active_reason():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler(lines).summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == pytest.approx(2070.0)
    assert out["sm_max_mhz"] == pytest.approx(2070.0)
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_hardware_slowdowns():
    lines = ["0, 1200, 2070, 800.0, 0x8, Active, Not Active, Active, Not Active"] * 3
    out = _sampler(lines).summary()
    assert out["sm_mhz"] == pytest.approx(1200.0)
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    out = _sampler([]).summary()
    assert out["samples"] == 0 and out["sm_mhz"] is None and out["reasons"] == []


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2070 MHz
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.fp32_peak_tflops(1035.0) == pytest.approx(bench.fp32_peak_tflops(2070.0) / 2)


def test_job_throughput_counts_every_replica():
    assert bench.job_throughput(1, 50, 100.0) == pytest.approx(500.0)
    assert bench.job_throughput(4, 50, 100.0) == pytest.approx(2000.0)
