"""The bench's reference arm (the oracle on the host cores) prints the contract's JSON
line; checked here on a tiny configuration of each amplitude mode (no GPU needed)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,amplitude", [("f6", "ta"), ("f6", "hk"), ("f3", "ta"), ("f9", "ta"),
                                               ("f9mlp", "ta")])
def test_reference_arm_json_line(workload, amplitude):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
           "--amplitude", amplitude, "--n-traj", "64", "--n-steps", "40", "--n-E", "32", "--cpu-sample", "8",
           "--steps", "1", "--warmup", "3"]
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


def test_clock_summary_reads_throttle_reasons():
    """The clock record beside every bench number: median SM clock, maximum clock and the
    throttle reasons seen active (from nvidia-smi's csv, noheader, nounits lines)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    c = bench.ClockSampler(0)
    c.lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "2040, 2070, 1200.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "truncated line",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append("1200, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 times the oracle and prints; the other ranks exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--n-traj", "64", "--n-steps", "40", "--n-E", "32", "--cpu-sample", "8"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
