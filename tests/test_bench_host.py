"""bench.py's host logic (no GPU): the clock record taken during the timed
region (median SM clock, throttle reasons seen as Active), the FP32 peak
derived from the unit counts, the whole-job throughput, the oracle arm's
isolation from the library, the shared config keys, and the staleness guard
of the ncu counters."""

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
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2070 MHz; the SM count is the device's
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.fp32_peak_tflops(1035.0) == pytest.approx(bench.fp32_peak_tflops(2070.0) / 2)
    assert bench.fp32_peak_tflops(2070.0, 76) == pytest.approx(bench.fp32_peak_tflops(2070.0) / 2)


def test_job_throughput_counts_every_replica():
    assert bench.job_throughput(1, 50, 100.0) == pytest.approx(500.0)
    assert bench.job_throughput(4, 50, 100.0) == pytest.approx(2000.0)


def test_oracle_arm_loads_no_part_of_the_library():
    """The reference arm builds its problem from the seeded generator alone:
    the ctypes binding (and with it libbs.so) is never imported."""
    import subprocess
    import sys
    code = ("import sys, bench; w, a, t = bench.workload_inputs(0); "
            "assert 'paper_2503_16424_gb300.bs' not in sys.modules, 'binding imported'; "
            "assert not any('libbs' in l for l in open('/proc/self/maps')), 'libbs.so mapped'; print('ok')")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=bench.ROOT, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_both_arms_report_the_same_config_keys():
    w, _, _ = bench.workload_inputs(0)
    one = bench.workload_config(w, 123, 1)
    assert one["n_gaussians"] == 262144 and one["n_pairs"] == 123
    assert set(one) == set(bench.workload_config(w, 5, 4))
    assert bench.workload_config(w, 5, 4)["parallelism"] == "independent images x4"


def test_ranks_get_independent_images():
    w0, a0, t0 = bench.workload_inputs(0)
    w1, a1, t1 = bench.workload_inputs(1)
    assert w0 == w1 and a0["open_ctrl"].shape == a1["open_ctrl"].shape
    assert not (a0["open_ctrl"] == a1["open_ctrl"]).all()


def test_host_cpu_reports_cores_and_a_model():
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_stale_counters_are_not_used():
    saved = dict(bench.NCU_CAPTURE)
    try:
        bench.NCU_CAPTURE.update(source_sha256_16="0" * 16,
                                 render_bwd_kernel={"flop_per_eval": 40.0, "dram_bytes": 1})
        r = bench.roofline(0.5, 1.0, 10, 10, 152, {"sm_max_mhz": 2070.0}, "measured")
        assert r["achieved"] is None and r["traffic"] is None and r["counters"].startswith("stale")
        bench.NCU_CAPTURE.update(source_sha256_16=bench.render_source_hash())
        r = bench.roofline(0.5, 1.0, 10 ** 9, 10 ** 9, 152, {"sm_max_mhz": 2070.0}, "measured")
        assert r["achieved"] == pytest.approx(40.0 * 1e9 / 1e-3 / 1e12, rel=1e-3) and r["traffic"] == 1
    finally:
        bench.NCU_CAPTURE.clear()
        bench.NCU_CAPTURE.update(saved)


def test_binning_launch_counts_follow_the_library_plan():
    """Kernels one binning call launches: the two-level sort where it applies
    (32-bit keys, at most 512 x 512 tiles), else key emission and the radix
    passes; the tile scan in one CTA when the counts fit its shared memory."""
    from paper_2503_16424_gb300 import bs
    # 2048^2, 16 px tiles, 262,144 Gaussians: 14 + 18 key bits, 128 x 128 tiles
    assert bench.binning_launches(bs.Canvas(2048, 2048, 16), 262144) == 4 + 7
    # 513 tile columns: the radix passes (2 of 7 bits), chunk owners and emission
    assert bench.binning_launches(bs.Canvas(4104, 64, 8), 6000) == 4 + 2 + 3 * 2 - 1
    # 64-bit keys on a 32768^2 canvas: radix passes, tile scan in three kernels
    assert bench.binning_launches(bs.Canvas(32768, 32768, 16), 1536) == 3 + 3 + 2 + 3 * 3 - 1
