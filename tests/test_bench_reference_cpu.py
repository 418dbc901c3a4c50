"""The bench's reference arm (the oracle timed on the host cores) keeps the
JSON-line contract: one line with the metric, a positive value, the unit and
direction of the headline, an e2e object without host-device traffic and a
cpu_baseline describing the sample it timed.  It needs no GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=240, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["metric"].startswith("l0 tuple-fits/sec at d=3")
    assert rec["unit"] == "tuple-fits/s" and rec["higher_is_better"] is True
    assert rec["value"] > 0 and rec["steps"] == 1 and rec["warmup"] == 1
    assert rec["config"]["workload"].startswith("C2:")
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"]
    assert "tuples" in cb["sample"]
