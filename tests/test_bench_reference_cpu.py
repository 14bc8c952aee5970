"""bench.py's reference arm runs the FP64 oracle on the host cores and prints
the contract's JSON line; checked here end to end on CPU (one timed step)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "block-applies/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "poisson_k8_eps1e-6_adaptive7"


@pytest.mark.slow
def test_oracle_on_all_cores_shares_one_sample():
    """bench.py's all-cores oracle timing: single-threaded processes released
    together, each on its own share of one random node order."""
    sys.path.insert(0, ROOT)
    import bench
    two = bench.run_oracle_parallel(2.0, 2)
    assert two["n_nodes"] == 7737 and two["items"] > 0 and two["seconds"] >= 2.0
    # every worker applies at least one chunk of 16 nodes of its share
    assert two["nodes"] >= 2 * 16
