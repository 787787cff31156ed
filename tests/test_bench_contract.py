"""bench.py's JSON line, checked on the arm that runs without a GPU: the
reference arm (the FP64 oracle on the host cores), on a two-string sample of
the default workload (the 4096-string modulated batch), and its
extrapolation from a sample to the whole workload."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--strings", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("4096 strings x 4 s")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_extrapolation_by_grid_point_updates():
    """A sample of the workload that runs at R updates/s gives the whole
    workload's samples/s at R; a sample equal to the workload gives its own
    rate back."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2311_18505_gb300 import workloads as W
    strings = W.batch_mixed(6, seconds=0.01, seed=2)
    n = strings[0]["n_samples"]
    total = sum(d["n_samples"] for d in strings)
    assert abs(bench.extrapolated_rate(strings, strings, n, 2.0) - total / 2.0) < 1e-9 * total
    sample = strings[:2]
    t = 0.5
    r = bench.extrapolated_rate(strings, sample, n, t)
    upd = sum(bench.oracle_cost(d, n) for d in sample) / t
    assert abs(r - total * upd / sum(bench.oracle_cost(d, n) for d in strings)) < 1e-9 * r
