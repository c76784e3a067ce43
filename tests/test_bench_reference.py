"""The reference arm of bench.py (the oracle timed on the host) on CPU: one JSON
line with the contract's keys, the oracle's own rate as value, cpu_baseline and
e2e describing the same run."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
                        "--cpu-seconds", "0.3", "--p", "2", "--n", "16"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_step_is_the_timed_step():
    """ms_per_step is the median time of one measured step (one oracle apply on
    the window), so steps x ms_per_step fits inside the run's own wall time."""
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "5", "--warmup", "3",
                        "--p", "2", "--n", "16"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][0])
    assert d["steps"] * d["ms_per_step"] * 1e-3 < wall
    assert d["config"]["window_n_dof"] / (d["ms_per_step"] * 1e-3) / 1e9 == pytest.approx(d["value"], rel=1e-3)


def test_all_cores_oracle_baseline():
    sys.path.insert(0, ROOT)
    import bench
    b = bench.oracle_baseline_all_cores(2, 16, 0.5, w=4)
    assert b["kind"] == "oracle" and b["cores"] == (os.cpu_count() or 1) and b["value"] > 0
