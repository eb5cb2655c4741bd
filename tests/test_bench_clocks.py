"""Host logic of the bench's clock record (no GPU, no nvidia-smi): which samples
describe the timed window, and which throttle reasons they report."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

LINE = "0, {sm}, 2070, 500.0, 0x0, {hw}, Not Active, Not Active, {pc}\n"


def _clk(samples, t0, t1):
    c = bench.Clocks(0)
    c.lines = [(t, LINE.format(sm=sm, hw=hw, pc=pc)) for t, sm, hw, pc in samples]
    c.t0, c.t1 = t0, t1
    return c.summary()


def test_samples_inside_the_window_are_used():
    s = _clk([(0.0, 1000, "Not Active", "Not Active"), (1.05, 2070, "Not Active", "Active"),
              (1.15, 2060, "Not Active", "Not Active"), (2.0, 900, "Active", "Not Active")],
             1.0, 1.2)
    assert s["samples"] == 2 and s["samples_in_window"] == 2
    assert s["sm_mhz"] == 2065.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]      # the samples outside are ignored


def test_short_window_takes_the_neighbouring_samples():
    s = _clk([(0.0, 1000, "Not Active", "Not Active"), (0.9, 2070, "Not Active", "Not Active"),
              (1.3, 2050, "Active", "Not Active")], 1.0, 1.02)
    assert s["samples"] == 2 and s["samples_in_window"] == 0
    assert s["sm_mhz"] == 2060.0 and s["reasons"] == ["hw_slowdown"]


def test_no_sampler_reports_no_samples():
    s = bench.Clocks(0).summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []
