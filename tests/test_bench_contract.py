"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the keys the benchmark contract fixes.  Runs on the CPU:
the oracle arm needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 1 and line["value"] > 0
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_committed_traffic_profile_matches_the_current_kernels():
    """bench.py reports the DRAM traffic of the committed ncu capture only
    while the stage kernels' sources hash to the value recorded with it; a
    kernel change must come with a new capture."""
    sys.path.insert(0, ROOT)
    import bench
    t = json.load(open(bench.TRAFFIC_FILE))
    assert t["kernel_source_hash"] == bench.kernel_source_hash()
    assert t["bytes_per_step"] == sum(t["dram_bytes_per_stage"])
    # at least the compulsory 112 B per stored cell and step of the staged RK4
    assert t["bytes_per_stored_cell_step"] >= 112.0
