"""bench.py's reference arm (the CPU oracle timed on the host cores) keeps the
JSON line contract: one line with impl "reference", the workload's metric and
unit, a cpu_baseline describing the run and an e2e object with no copies."""
import json
import os
import subprocess
import sys

import pytest


@pytest.mark.timeout(300)
@pytest.mark.parametrize("workload", ["plain_64k", "pbr_1m"])
def test_reference_arm_json_line(workload):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", workload,
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=280, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
