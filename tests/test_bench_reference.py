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


def test_scalar_floor_counts_adjacent_swaps():
    """The bench's unblocked floor F_min = 12 n flops per adjacent swap.  For
    1x1 blocks the swaps are the (unselected above selected) pairs: the
    oracle's swap count equals that brute-force count, and over a random
    selection of a fraction p, F_min is about 6 p (1 - p) n^3."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    rng = np.random.default_rng(3)
    n = 60
    S = np.asfortranarray(np.triu(rng.standard_normal((n, n)), 1) + np.diag(np.arange(n) + 1.0))
    sel = (rng.random(n) < 0.4).astype(np.int32)
    pairs = sum(1 for i in range(n) for j in range(i + 1, n) if not sel[i] and sel[j])
    r = oracle.reorder(S, None, sel)
    assert r["status"] == 0 and r["nswaps"] == pairs
    assert bench.f_min_flops(n, pairs) == 12.0 * n * pairs
    n, p = 4000, 0.35
    s = rng.random(n) < p
    inv = int(np.sum(np.cumsum(~s)[s]))
    assert abs(bench.f_min_flops(n, inv) / (6 * p * (1 - p) * n ** 3) - 1) < 0.05
