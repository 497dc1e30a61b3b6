"""The benchmark's reference arm (the CPU oracle on the host cores) prints one
well-formed JSON line; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "n8", "--steps", "2", "--warmup", "1", "--cpu-seconds", "0.2")
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "steps/s" and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # each step of this arm is one bounded sample: steps x ms_per_step is the time the samples took
    assert "step_kind" in d and 0 < d["ms_per_step"] < 60e3
    assert d["steps"] * d["ms_per_step"] * 1e-3 < 120


def test_reference_arm_without_oracle_form():
    d = _run("--impl", "reference", "--workload", "grad")
    assert d["impl"] == "reference" and "unavailable" in d
