"""The benchmark's clock record: samples inside the timed window only, the
throttle reasons seen there, and the fallbacks when the window is shorter than
the sampling interval or the lines carry no usable timestamp."""
import datetime

import bench


def _line(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), "2070", "800.0", "0x0"] + list(reasons))


def test_samples_inside_the_window():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.1, 1000), _line(t0 + 0.01, 2070), _line(t0 + 0.03, 2060),
             _line(t0 + 0.05, 2050, ("Not Active", "Not Active", "Not Active", "Active")), _line(t0 + 0.2, 900)]
    s = bench.summarize_clock_lines(lines, t0, t0 + 0.06)
    assert s["window"] == "during" and s["samples"] == 3
    assert s["sm_mhz"] == 2060 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_short_window_takes_the_nearest_sample():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.5, 1500), _line(t0 + 0.012, 2070), _line(t0 + 0.5, 1200)]
    s = bench.summarize_clock_lines(lines, t0 + 0.001, t0 + 0.005)
    assert s["window"] == "nearest" and s["samples"] == 1 and s["sm_mhz"] == 2070


def test_lines_without_timestamps_and_garbage():
    lines = ["bad line", "x, 0, 2070, 2070, 1.0, 0x0, Not Active, Active, Not Active, Not Active",
             "y, 0, notanumber, 2070, 1.0, 0x0, a, b, c, d"]
    s = bench.summarize_clock_lines(lines, 1.0, 2.0)
    assert s["window"] == "untimed" and s["samples"] == 1
    assert s["reasons"] == ["hw_thermal_slowdown"]
    assert bench.summarize_clock_lines([], 1.0, 2.0) is None
