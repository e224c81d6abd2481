"""The reference arm of bench.py (the CPU oracle timed on a bounded sample of
the 2049^2 workload) runs without a GPU and prints one JSON line in the
benchmark's format: same metric and unit as the GPU arm, the oracle described
as the CPU baseline, and an end-to-end entry with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-budget", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    assert r["metric"] == r["unit"] == "local sample-solves/s" and r["higher_is_better"] is True
    assert r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 0 and r["n_gpus"] == 1
    assert r["config"]["workload"] == "elliptic-2049-lognormal-32x32-b16-S128"
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
