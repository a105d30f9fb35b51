"""The benchmark's reference arm (the CPU oracle timed on the host cores) prints one JSON line
with the contract's keys, for the headline metric and for the DQMC mode, on a small workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("mode,unit", [("step", "evals/s"), ("dqmc", "chain-sweeps/s")])
def test_reference_arm_prints_contract_line(mode, unit):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--mode", mode,
                          "--workload", "holstein_4x4_L40", "--steps", "1", "--warmup", "0", "--nsweeps", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == unit and line["value"] > 0.0
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
                "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "holstein_4x4_L40"
