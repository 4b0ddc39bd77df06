"""Host-side pieces of bench.py's measurement: the roofline's peak (the measured copy bandwidth
from MEASURED_PEAKS.json, else the stated fallback) and the clock summary taken from
nvidia-smi rows (median SM clock under load, the maximum, and every throttle reason that
was active in any sample)."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_peak_is_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6784.5, "bf16_tflops": 1940.6}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6784.5, "measured")


@pytest.mark.parametrize("content", [None, "not json", json.dumps({"bf16_tflops": 1940.6}),
                                     json.dumps({"hbm_gbs": "fast"})])
def test_peak_falls_back_when_no_measured_bandwidth(tmp_path, monkeypatch, content):
    if content is not None:
        (tmp_path / "MEASURED_PEAKS.json").write_text(content)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")


def row(sm, mx, reasons=()):
    """One nvidia-smi CSV row in the sampler's field order (index, sm, max sm, power, active,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ["0", str(sm), str(mx), "900.5", "0x0000000000000004" if reasons else "0x0"] + flags


def test_clock_summary_takes_the_median_and_every_active_reason():
    s = bench.ClockSampler()
    s.rows = [row(2070, 2070), row(1995, 2070, ["sw_power_cap"]), row(2032, 2070),
              row(1800, 2070, ["hw_slowdown"])]
    got = s.summary()
    assert got["sm_mhz"] == pytest.approx((1995 + 2032) / 2)
    assert got["sm_max_mhz"] == 2070
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert got["samples"] == 4


def test_clock_summary_skips_unreadable_fields_and_reports_no_samples():
    s = bench.ClockSampler()
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    s.rows = [["0", "[N/A]", "[N/A]", "[N/A]", "0x0"], row(2070, 2070)]
    got = s.summary()
    assert got["sm_mhz"] == 2070 and got["sm_max_mhz"] == 2070 and got["reasons"] == [] and got["samples"] == 2
