"""The sweep oracle's pins must catch plausible mistakes: each case plants
one (a wrong sign, a dropped term, a transposed application, the wrong
order of the bulges in a step, a shortened row range) in a temporary copy
of `oracle/sweep_oracle.c` and runs the pins of
tests/test_oracle_sweep.py against it in a subprocess."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sweep_oracle.c")

MUTANTS = [
    ("introduction x0 sign", "x[0] = h00 * h00 + h01 * h10 - s * h00 + p;",
     "x[0] = h00 * h00 + h01 * h10 + s * h00 + p;"),
    ("introduction x1 term dropped", "x[1] = h10 * (h00 + h11 - s);", "x[1] = h10 * (h00 - s);"),
    ("introduction x2 wrong entry", "x[2] = h10 * h21;", "x[2] = h01 * h21;"),
    ("shift product sign", "sr[2 * b] * sr[2 * b + 1] - si[2 * b] * si[2 * b + 1]",
     "sr[2 * b] * sr[2 * b + 1] + si[2 * b] * si[2 * b + 1]"),
    ("bulges top first", "for (int b = 0; b < nb; ++b) {\n            const int k = tau - 3 * b - 1;",
     "for (int b = nb - 1; b >= 0; --b) {\n            const int k = tau - 3 * b - 1;"),
    ("right rows shortened", "const int rend = (k + 5 < n) ? k + 5 : n;",
     "const int rend = (k + 4 < n) ? k + 4 : n;"),
    ("column update transposed", "for (int i = 0; i < len; ++i) w += EL(H, ldH, r, r0 + i) * v[i];",
     "for (int i = 0; i < len; ++i) w += EL(H, ldH, r0 + i, r) * v[i];"),
    ("reflector sign", "double b = alpha >= 0.0 ? -norm : norm;", "double b = alpha >= 0.0 ? norm : -norm;"),
    ("last bulge stops early", "const int last = (n - 3) + 3 * (nb - 1) + 1;",
     "const int last = (n - 3) + 3 * (nb - 1);"),
    ("introduction misses row 3", "apply(n, H, ldH, Q, ldQ, 0, 3, v, tau, 0, n < 4 ? n : 4);",
     "apply(n, H, ldH, Q, ldQ, 0, 3, v, tau, 0, n < 3 ? n : 3);"),
    ("bulge fill not cleared", "for (int i = 1; i < len; ++i) EL(H, ldH, k + 1 + i, k) = 0.0;",
     "for (int i = 1; i < 1; ++i) EL(H, ldH, k + 1 + i, k) = 0.0;"),
    ("Q not updated", "            for (int i = 0; i < len; ++i) EL(Q, ldQ, r, r0 + i) -= w * v[i];",
     "            for (int i = 0; i < len; ++i) (void)w;"),
]

BATTERY = r"""
import sys, numpy as np
sys.path.insert(0, ROOT)
import oracle
oracle._lib = oracle.load(SO)
from tests import test_oracle_sweep as P
checks = [
    lambda: [P.test_implicit_q_theorem(n, ns, tol) for n, ns, tol in [(12, 2, 1e-14), (12, 4, 1e-13), (20, 6, 1e-13)]],
    lambda: [P.test_invariants(n, ns) for n, ns in [(4, 2), (9, 4), (60, 8)]],
    lambda: P.test_exact_shifts_deflate(),
    lambda: P.test_two_by_two_pair_closed_form(),
]
failed = 0
for c in checks:
    try:
        with np.errstate(all="ignore"):
            c()
    except Exception:
        failed += 1
print("FAILED_CHECKS", failed)
sys.exit(1 if failed else 0)
"""


def build(src, out):
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-o", out,
                    os.path.join(ROOT, "oracle", "reorder_oracle.c"), src, "-lm"], check=True)
    return out


def run_battery(so):
    code = BATTERY.replace("ROOT", repr(ROOT)).replace("SO", repr(so))
    try:
        p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=300, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return 124, "timeout"
    return p.returncode, p.stdout + p.stderr


def test_battery_passes_on_oracle(tmp_path):
    rc, out = run_battery(build(SRC, str(tmp_path / "orig.so")))
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_killed(name, old, new, tmp_path):
    with open(SRC) as f:
        src = f.read()
    assert old in src, f"mutation anchor for {name!r} not found"
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    rc, out = run_battery(build(str(c), str(tmp_path / "mut.so")))
    assert rc != 0, f"mutant {name!r} survived the pins"
