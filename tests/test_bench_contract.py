"""The bench's reference arm (the oracle on the host cores) prints the contract's JSON
line; checked here on a tiny configuration of each amplitude mode (no GPU needed)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("amplitude", ["ta", "hk"])
def test_reference_arm_json_line(amplitude):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--amplitude", amplitude,
           "--n-traj", "64", "--n-steps", "40", "--n-E", "32", "--cpu-sample", "8", "--steps", "1", "--warmup", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "trajectory-steps/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert ("Herman-Kluk" in d["config"]["workload"]) == (amplitude == "hk")


def test_reference_arm_reports_unavailable_workloads():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "batch"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and "unavailable" in d
