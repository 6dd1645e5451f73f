"""Host logic of the benchmark's output on the CPU: the final line is strict
JSON (no NaN or Infinity), short, and holds exactly the headline keys; the
stats cadence times at least one stats call in any run; the clock summary
keeps the samples of the timed region."""
import json
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _strict(s):
    def bad(c):
        raise ValueError(f"non-standard JSON constant {c}")
    return json.loads(s, parse_constant=bad)


def test_non_finite_floats_become_null():
    stats = {"volume": 1.0, "energy": float("nan"), "phi_min": -float("inf"),
             "nested": [np.float64("nan"), np.float32(2.5), (np.int64(3), float("inf"))]}
    s = bench.dumps({"leg": "last_stats", **stats})
    d = _strict(s)
    assert d["energy"] is None and d["phi_min"] is None
    assert d["nested"] == [None, 2.5, [3, None]]
    assert d["volume"] == 1.0


def test_headline_line_is_short_and_strict():
    """A line as run_gpu builds it, with a stats record holding NaN and a long
    leg list: the headline keeps only its keys and stays under 2 KB."""
    args = bench.parse(["--steps", "20", "--warmup", "5"])
    w = bench.workload(args)
    line = {"metric": bench.METRIC, "value": 6.0e11, "unit": bench.UNIT, "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 0.22, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": bench.arm_config(args, w, 1),
            "roofline": {"bound": "hbm", "achieved": 5100.0, "peak": 6785.2, "unit": "GB/s", "frac": 0.75,
                         "peak_kind": "measured", "frac_of_nominal": 0.64, "traffic": 1.02e9,
                         "kernel": "spfm_step_kernel", "bytes_per_update": 8, "avg_launch_ms": 0.211,
                         "timed": "stencil kernel, which writes the periodic ghost images itself; "
                                  "events around 20-step chunks"},
            "cpu_baseline": {"value": 2.1e8, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                             "sample": "3 FP64 oracle steps on a 512x512x40 z-slab of the workload (12.0 s)"},
            "e2e": {"value": 4e11, "unit": bench.UNIT, "h2d_bytes_per_step": 1.1e7, "d2h_bytes_per_step": 1.1e7,
                    "note": "per call: host field in, 50 steps, stats, host field out"},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "power_w_max": float("nan"), "reasons": [],
                       "samples": 3, "window": "timed region"},
            "gpu_launches": 22, "stats_call": {"ms": 0.44, "calls": 1, "every": 20, "note": "x"},
            "legs": ["last_stats", "grain_sphericity", "variants", "bf16_storage", "tilted_256",
                     "shape_relaxation", "friction_1d", "force_oscillation", "kinetic_anisotropy",
                     "batched", "serving", "velocity_vs_oracle"],
            "batched": {"rows": list(range(1000))}, "last_stats": {"energy": float("nan")}}
    h = bench.headline(line)
    assert set(h) <= set(bench.HEADLINE_KEYS)
    assert "batched" not in h and "last_stats" not in h
    s = bench.dumps(h)
    assert len(s) < 2048, len(s)
    d = _strict(s)
    assert d["clocks"]["power_w_max"] is None
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["roofline"]["frac"] == pytest.approx(d["roofline"]["achieved"] / d["roofline"]["peak"], rel=0.01)


@pytest.mark.parametrize("steps,every", [(1, 1), (20, 20), (50, 50), (3000, 50), (51, 50)])
def test_stats_cadence_times_at_least_one_call(steps, every):
    assert bench.stats_cadence(steps) == every
    assert steps // bench.stats_cadence(steps) >= 1


def test_clock_summary_keeps_the_timed_region():
    lines = [
        "2026/12/04 10:00:00.000, 0, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "2026/12/04 10:00:00.500, 0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Active\n",
        "2026/12/04 10:00:00.600, 0, 2040, 2070, 720.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "2026/12/04 10:00:02.000, 0, 1100, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "garbage\n",
    ]
    import datetime
    t0 = datetime.datetime(2026, 12, 4, 10, 0, 0, 450000).timestamp()
    t1 = datetime.datetime(2026, 12, 4, 10, 0, 0, 650000).timestamp()
    rows, inside = bench.ClockSampler.parse_rows(lines, (t0, t1), 0.0)
    assert inside and len(rows) == 2
    d = bench.ClockSampler.summarise(rows, inside)
    assert d["sm_mhz"] == pytest.approx(2055.0) and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["sw_power_cap"] and d["window"] == "timed region"
    rows, inside = bench.ClockSampler.parse_rows(lines)
    assert not inside and len(rows) == 4
    assert bench.ClockSampler.summarise([], False)["samples"] == 0
    assert math.isfinite(bench.ClockSampler.summarise(rows, inside)["power_w_max"])
