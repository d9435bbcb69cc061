"""Host logic of bench.py (no GPU): the reference arm's JSON line, the roofline and rate
arithmetic, the clock sampler's reading of nvidia-smi lines, and the percentiles."""
import json
import math

import pytest

import bench

CONTRACT_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config"}


class _Args:
    steps = 1
    warmup = 0


def test_reference_arm_line_keeps_the_contract():
    out = bench.run_reference(_Args(), 0, 1)
    json.dumps(out)                                   # one JSON line
    assert CONTRACT_KEYS <= set(out)
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["higher_is_better"] is True and out["vs_baseline"] is None
    assert out["value"] > 0 and math.isclose(out["ms_per_step"], 1e3 / out["value"], rel_tol=1e-9)
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    # the same workload description as the GPU arm's line
    w, _, _ = bench.workload_inputs()
    ours = bench.workload_config(w, "mixed", "flushed", "replicas x1")
    assert set(out["config"]) == set(ours)
    same = {k for k in ours if k not in ("precision", "l2", "parallelism")}
    assert all(out["config"][k] == ours[k] for k in same)


def test_rate_against_hbm_and_alu_peaks():
    pk = {"hbm_gbs": 5000.0, "sm_max_mhz": 2000.0}
    r = bench.rate("coarse_project", 2.0, 10e9 * 2e-3, 0.0, pk, "measured")   # 10 GB/s-equivalent bytes in 2 ms
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(10.0) and r["frac"] == pytest.approx(10.0 / 5000.0)
    peak = 152 * 128 * 2 * 2000e6 / 1e12
    r = bench.rate("leaf_sweep", 1.0, 0.0, 3e9, pk, "measured")               # 3 TFLOP/s
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(peak) and r["achieved"] == pytest.approx(3.0)
    r = bench.rate("svd", 1.0, 1.0, 1.0, pk, "measured")
    assert r["achieved"] is None and r["frac"] is None


def test_roofline_uses_the_timed_category_and_the_profiled_share():
    pk = {"hbm_gbs": 4000.0}
    prof = {"coarse_project": (1.0, 10, 4e9 * 1e-3, 0.0)}
    prof_all = {"coarse_project": (3.0, 20, 0.0, 0.0), "leaf_sweep": (1.0, 5, 0.0, 0.0)}
    r = bench.roofline(None, prof, prof_all, "coarse_project", pk, "measured")
    assert r["launches"] == 10 and r["avg_launch_ms"] == pytest.approx(0.1)
    assert r["achieved"] == pytest.approx(4.0) and r["frac"] == pytest.approx(1e-3)
    assert r["share_of_profiled_ms"] == pytest.approx(0.75)
    assert r["alg_bytes_per_launch"] == pytest.approx(4e6 / 10)
    assert r["traffic"] == bench.TRAFFIC_BYTES_PER_LAUNCH.get("coarse_project")
    assert bench.roofline(None, {}, prof_all, "coarse_project", pk, "measured") is None


def test_clock_sampler_reads_reasons_and_median():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active",
        "garbage line",
    ]
    out = s.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_percentiles():
    assert bench.pct([], 50) is None
    assert bench.pct([3.0, 1.0, 2.0], 50) == 2.0
    assert bench.pct([1.0, 2.0], 99) == pytest.approx(1.99)
