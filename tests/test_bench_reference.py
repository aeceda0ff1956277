"""bench.py's reference arm (the CPU oracle timed on the host cores) keeps
the JSON-line contract for the next rows' workloads, and ranks other than 0
exit quietly (runs without a GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                       text=True, timeout=600, cwd=ROOT, env=e)
    assert p.returncode == 0, p.stderr[-2000:]
    return p.stdout


@pytest.mark.parametrize("workload,unit", [("h4000", "shifts/s"), ("g4000", "eigs/s")])
def test_reference_line(workload, unit):
    out = run_bench("--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "0")
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == unit
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == workload
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0
    assert e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_exit_quietly():
    out = run_bench("--impl", "reference", "--workload", "h4000", "--steps", "1", "--warmup", "0",
                    env={"RANK": "1", "WORLD_SIZE": "2"})
    assert out.strip() == ""
