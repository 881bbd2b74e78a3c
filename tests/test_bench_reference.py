"""The reference arm of bench.py (the CPU oracle timed on a bounded sample of
the workload) runs without a GPU and prints the contract's JSON line with the
same metric as the workload's own arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,metric", [
    ("tiny", "decompressed GB/s device-resident"),
    ("fastq", "decompressed GB/s device-resident"),
    ("encode", "encoded input GB/s, input resident in device memory"),
])
def test_reference_arm_line(workload, metric):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
                        "--size", "3000000", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == metric and line["unit"] == "GB/s"
    assert line["value"] > 0 and line["steps"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
