"""The benchmark's clock summary (nvidia-smi samples taken during the timed
region): median SM clock, maximum, and every throttle reason seen active,
parsed from the CSV nvidia-smi writes. CPU only (a recorded sample file)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def summary_of(tmp_path, lines):
    cs = bench.ClockSampler(0)
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    cs.path = str(path)
    cs.proc = object()  # a sampler that ran
    return cs.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = summary_of(tmp_path, rows)
    assert s["sm_mhz"] == 2010.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_clock_summary_reports_thermal_and_hw_slowdown(tmp_path):
    rows = [
        "0, 1500, 2070, 1000.0, 0x48, Active, Not Active, Active, Not Active",
        "0, 1400, 2070, 1000.0, 0x48, Not Active, Active, Not Active, Not Active",
    ]
    s = summary_of(tmp_path, rows)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1450.0


def test_clock_summary_without_sampler():
    cs = bench.ClockSampler(0)
    s = cs.summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_measured_peaks_are_read():
    gbs, src = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and gbs > 1000.0
    else:
        assert src == "fallback" and gbs == 6800.0
