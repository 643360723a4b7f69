"""Host logic of bench.py that needs no GPU: the clock record built from
nvidia-smi rows (median SM clock, maximum, throttle reasons seen, malformed
rows skipped) and the per-workload default step counts."""
import sys

import bench


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, pcap]


def test_clock_summary():
    s = bench.ClockSampler(0)
    s.rows = [_row(2070, 2070), _row(2040, 2070, pcap="Active"), _row(2070, 2070), ["garbage"],
              _row("[N/A]", 2070)]
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_throttling():
    s = bench.ClockSampler(0)
    s.rows = [_row(1500, 2070, hwt="Active"), _row(1400, 2070, swt="Active"), _row(1600, 2070, hw="Active")]
    out = s.summary()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_default_steps(monkeypatch):
    for argv, steps in ([[], 5], [["--workload", "pt27"], 50], [["--workload", "batch16"], 5],
                        [["--impl", "reference"], 3], [["--steps", "7"], 7]):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        assert bench.parse().steps == steps
