"""bench.py's host logic on the CPU: the clock record that decides whether a
timed run is kept, the workloads' eps recipes and the peak lookup."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
LINE = "0, {sm}, 2070, 900.5, 0x0000000000000000, {hw}, Not Active, {swt}, {cap}"


def _line(sm=2070, hw="Not Active", swt="Not Active", cap="Not Active"):
    return LINE.format(sm=sm, hw=hw, swt=swt, cap=cap)


def test_clock_record_median_and_reasons():
    lines = [_line(2070), _line(2055), _line(1980, cap="Active"), "garbage", "0, N/A, 2070, 1, 0, a, b, c, d"]
    r = bench.parse_clock_lines(lines)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_slowdowns():
    r = bench.parse_clock_lines([_line(hw="Active"), _line(swt="Active"), _line()])
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples():
    r = bench.parse_clock_lines([])
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == ["no samples"]


def test_workload_eps_recipes():
    for name, wl in bench.WORKLOADS.items():
        e = bench.workload_eps(wl, 500)
        assert e.shape == (500,) and np.all((e > 0) & (e < 1)), name
        np.testing.assert_array_equal(e, bench.workload_eps(wl, 500))  # seeded
        spec = wl["eps"]
        if isinstance(spec, float):
            assert np.all(e == spec)
        elif spec[0] == "uniform":
            assert np.all((e >= spec[1]) & (e <= spec[2])) and len(np.unique(e)) > 400
            assert not np.array_equal(e, bench.workload_eps(wl, 500, rank=1))  # ranks draw their own
        else:
            assert set(np.unique(e)) <= set(spec[1:])


def test_peak_lookup_reads_measured_file():
    hbm, kind = bench.load_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert hbm == json.load(f)["hbm_gbs"] and kind == "measured"
    else:
        assert (hbm, kind) == (6800.0, "fallback")
