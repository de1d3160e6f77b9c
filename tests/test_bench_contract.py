"""bench.py's algorithmic-work constants equal the oracle's count, and the
reference arm prints the contract's JSON line (CPU only)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_constants_match_oracle_count(oracle_mod):
    sys.path.insert(0, ROOT)
    import bench
    from oracle import count_work
    w = count_work.work()
    assert bench.ALGO["fp64_flops_per_subgrid_stage"] == w["fp64_flops_per_subgrid_stage"]
    assert bench.ALGO["bytes_per_subgrid_stage"] == w["bytes_per_subgrid_stage"]


@pytest.mark.slow
def test_reference_arm_json_line(oracle_mod):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "cpu_baseline", "e2e", "config", "higher_is_better"):
        assert k in line
