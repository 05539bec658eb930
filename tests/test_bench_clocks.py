"""The clock summary of bench.py on CPU: of nvidia-smi's timestamped samples only those
inside the timed region count, throttle reasons seen there are reported, and a region
shorter than the sampling period takes the sample nearest to its middle."""
import os
import sys
from datetime import datetime

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts, sm, mx, hw="Not Active", cap="Not Active"):
    stamp = datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return "%s, %d, %d, 900.5, %s, Not Active, Not Active, %s" % (stamp, sm, mx, hw, cap)


def test_only_samples_inside_the_region_count():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 1.0, 1200, 2070, hw="Active"),   # before: a slowdown not in the region
             _line(t0 + 0.05, 2070, 2070),
             _line(t0 + 0.15, 2055, 2070, cap="Active"),
             _line(t0 + 0.25, 2070, 2070),
             _line(t0 + 2.0, 300, 2070)]                   # after: idle clock
    r = bench.Clocks.summarize(lines, t0, t0 + 0.3)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert abs(r["region_s"] - 0.3) < 1e-9


def test_short_region_takes_the_nearest_sample():
    t0 = 1_800_000_000.0
    lines = [_line(t0 - 0.5, 2070, 2070), _line(t0 + 0.6, 1965, 2070, hw="Active")]
    r = bench.Clocks.summarize(lines, t0 + 0.3, t0 + 0.32)
    assert r["samples"] == 1 and r["sm_mhz"] == 1965.0 and r["reasons"] == ["hw_slowdown"]


def test_unparsable_output_gives_none():
    assert bench.Clocks.summarize(["No devices were found"], 0.0, 1.0) is None
