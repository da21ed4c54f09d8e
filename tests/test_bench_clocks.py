"""bench.py's clock record on CPU: samples are stamped on the host and the summary keeps
those inside the timed window, falls back to the samples around it when the window held
none (and says so), and reports the throttle reasons a sample shows as active."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

ROW = "0, {mhz}, 2070, 1000, 0x0, Not Active, {hw_th}, Not Active, {pcap}"


def _sampler(lines, t0=10.0, t1=10.01):
    c = bench.ClockSampler(0)
    c.t0, c.t1 = t0, t1
    c.lines = lines
    return c


def test_summary_keeps_the_timed_window():
    c = _sampler([(9.7, ROW.format(mhz=900, hw_th="Not Active", pcap="Not Active")),
                  (10.004, ROW.format(mhz=2070, hw_th="Not Active", pcap="Active")),
                  (10.2, ROW.format(mhz=1200, hw_th="Active", pcap="Not Active"))])
    s = c.summary()
    assert s["window"] == "timed region" and s["samples"] == 1
    assert s["sm_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


def test_summary_falls_back_to_the_samples_around_a_short_window():
    c = _sampler([(9.7, ROW.format(mhz=2000, hw_th="Not Active", pcap="Not Active")),
                  (10.3, ROW.format(mhz=2050, hw_th="Active", pcap="Not Active")),
                  (11.0, ROW.format(mhz=100, hw_th="Not Active", pcap="Not Active"))])
    s = c.summary()
    assert s["window"].startswith("within 0.5 s") and s["samples"] == 2
    assert s["sm_mhz"] == 2025 and s["reasons"] == ["hw_thermal_slowdown"]


def test_no_samples_no_record():
    assert _sampler([]).summary() is None
    assert _sampler([(10.005, "garbled")]).summary() is None
