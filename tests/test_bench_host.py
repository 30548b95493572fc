"""Host logic of the benchmark (no GPU): kernels counted per find, the
measured peak, the traffic taken from the committed profile only while the
kernel sources match it, and the clock-sample parsing that rejects
throttled runs."""
import json
import os

import bench


def test_kernels_per_find():
    for m in (4, 7):
        assert bench.kernels_per_find(m, None) == 3        # dense pass, tile scan, copy
    for m in (8, 16, 64):
        assert bench.kernels_per_find(m, None) == 2        # count pass (+ tile scan), placement
    assert bench.kernels_per_find(16, {"layout": 1}) == 1  # single-pass find
    assert bench.kernels_per_find(8, {"layout": 1}) == 3
    assert bench.kernels_per_find(4, {"layout": 2}) == 1
    assert bench.kernels_per_find(4, {"layout": 4}) == 2


def test_measured_peak_and_config():
    peak, kind = bench.measured_peak_hbm()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == json.load(open(path))["hbm_gbs"]
    else:
        assert kind == "fallback"
    c = bench.config_dict(bench.TEXT_BYTES, 1, None)
    assert c["workload"] and c["text_bytes"] == 3_200_000_000 and c["patterns"] == [4, 8, 16, 32, 64]


def test_traffic_only_for_the_profiled_sources(monkeypatch):
    t = bench.profiled_traffic()
    assert t is None or t > bench.TEXT_BYTES                # bytes of a whole find
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 16)
    assert bench.profiled_traffic() is None


def test_clock_parsing_flags_throttling():
    cs = bench.ClockSampler("0")
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2070, 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active",
                "garbage line"]
    r = cs.stop()
    assert r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["sm_mhz"] == 2070.0
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
