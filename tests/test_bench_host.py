"""Host-side parts of bench.py without a GPU: the clock record that decides whether a
run is kept, the roofline peak, and the rule that profiled DRAM traffic is reported only
for the kernel sources it was captured on."""
import json
import os

import bench


def _sample(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", hw, hwt, swt, cap]


def test_clock_summary_takes_the_median_and_collects_active_reasons():
    c = bench.ClockSampler()
    c.samples = [_sample(2070, 2070), _sample(1980, 2070, cap="Active"), _sample(2070, 2070),
                 _sample(1500, 2070, hwt="Active")]
    s = c.summary()
    assert s["sm_mhz"] == 2025.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_says_so():
    s = bench.ClockSampler().summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["unsampled"]


def test_peak_is_the_measured_copy_bandwidth_else_the_fallback():
    peak, kind = bench._peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            assert kind == "measured" and peak == float(json.load(fh)["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_profiled_traffic_only_for_the_sources_it_was_captured_on(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    key = "rb_4096x2048_fp32"
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: d[key]["source_hash"])
    assert bench._profiled_traffic(key) == d[key]["read"] + d[key]["write"] == d[key]["bytes_per_launch"]
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "0" * 16)
    assert bench._profiled_traffic(key) is None
    assert bench._profiled_traffic("no_such_workload") is None
