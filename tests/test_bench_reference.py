"""The reference arm of bench.py (the CPU oracle on the workload graph) runs
without a GPU and prints one JSON line with the contract's keys."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
         "--workload", "er2000", "--h", "2", "--steps", "1", "--warmup", "0"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["host"]["nproc"] >= 1
    assert line["config"]["same_config"] is True and "full workload" in line["config"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
