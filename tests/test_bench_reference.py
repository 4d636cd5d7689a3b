"""The benchmark's reference arm (the oracle timed on the host cores) keeps
the line format the benchmark reports: one JSON line with the metric, unit
and direction of the GPU line, a `cpu_baseline` describing the run and an
`e2e` object with no host-device bytes; ranks other than 0 print nothing.
Runs on the CPU (the arm needs no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None):
    e = dict(os.environ)
    if env:
        e.update(env)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=e)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


@pytest.mark.parametrize("workload", ["amr2_base64", "batching_base128"])
def test_reference_arm_line(workload):
    lines = _run(["--impl", "reference", "--workload", workload, "--steps", "1",
                  "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Mcell/s of Jv+V-cycle" and d["unit"] == "Mcell/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    lines = _run(["--impl", "reference", "--workload", "amr2_base64", "--steps", "1",
                  "--warmup", "1"], env={"RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []
