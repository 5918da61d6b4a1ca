"""The reference arm of bench.py (the oracle with the paper's solver design on the
host cores) prints one JSON line with the contract's keys; run on the small c1
beam so that it takes seconds.  Its steps (one subdomain each) run
concurrently, one per core."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c1",
                          "--steps", "3", "--warmup", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True).stdout
    line = json.loads([x for x in out.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "subdomains/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["steps"] == 3 and line["warmup"] == 2
    # the three timed subdomains run concurrently (one round on this machine's cores)
    assert line["cpu_baseline"]["cores"] == min(3, os.cpu_count() or 1)
