"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index,
a transposed operand) in a temporary copy of the oracle's C source,
compiles it on the CPU, and runs a battery of the pins against it in a
subprocess.  The battery must fail for every mutant and pass for the
unmodified source.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text to find, replacement); the first occurrence is replaced.
MUTANTS = [
    ("rotation sign on rows", "EL(A, ld, i + 1, k) = c * y - s * x;",
     "EL(A, ld, i + 1, k) = c * y + s * x;"),
    ("givens angle sign", "double c = t12 / h, s = (t22 - t11) / h;",
     "double c = t12 / h, s = (t11 - t22) / h;"),
    ("1x1 swap drops Q update", "if (Q) rot_cols(Q, ldQ, j, 0, n, c, s);\n        /* new block",
     "/* new block"),
    ("sylvester T22 transposed", "if (i == l) v -= EL(T22, ld22, m, k);",
     "if (i == l) v -= EL(T22, ld22, k, m);"),
    ("sylvester T11 sign", "if (k == m) v += EL(T11, ld11, i, l);",
     "if (k == m) v -= EL(T11, ld11, i, l);"),
    ("householder tau", "*tau = (beta - alpha) / beta;", "*tau = (alpha - beta) / beta;"),
    ("complement vector transposed", "double u[3] = {gamma, X[0], X[2]};",
     "double u[3] = {gamma, X[2], X[0]};"),
    ("weak test dropped", "if (lower > thresh) return 1;", "if (lower > 1e300) return 1;"),
    ("strong test sign", "double e = fabs(E[c * 4 + r] - D[c * 4 + r]);",
     "double e = fabs(E[c * 4 + r] + D[c * 4 + r]);"),
    ("column update misses a row", "house_cols(S, ldS, j, len1, v1, tau1, 0, j);",
     "house_cols(S, ldS, j, len1, v1, tau1, 1, j);"),
    ("second reflector skipped", "house_rows(S, ldS, j + 1, 3, v2, tau2, j + k, n);",
     "(void)0;"),
    ("diagonal not equalized", "n11 = avg;\n        n22 = avg;", "n11 = avg;"),
    ("standardization angle", "double sin2 = -sg * 2.0 * p / r2;",
     "double sin2 = sg * 2.0 * p / r2;"),
    ("real split uses wrong root", "double x1 = p >= 0.0 ? p + r : p - r;",
     "double x1 = p >= 0.0 ? p - r : p + r;"),
    ("block above assumed 1x1", "int pa = (here - 2 >= ks && EL(S, ldS, here - 1, here - 2) != 0.0) ? 2 : 1;",
     "int pa = 1;"),
    ("2x2 selection not merged", "sel[j] = sel[j + 1] = s2;", "(void)s2;"),
    ("abort ignored", "if (!ok && abort_on_reject) break;", "if (!ok && abort_on_reject < 0) break;"),
    ("selection flags left behind", "for (int i = j; i < j + q; ++i) sel[i] = 1;\n",
     "for (int i = j; i < j; ++i) sel[i] = 1;\n"),
    ("eigenvalue imaginary part", "double im = sqrt(fabs(EL(S, ldS, j, j + 1))) * sqrt(fabs(EL(S, ldS, j + 1, j)));",
     "double im = sqrt(fabs(EL(S, ldS, j, j + 1)));"),
]

BATTERY = r"""
import sys, numpy as np
sys.path.insert(0, ROOT)
import oracle
from tests import test_oracle_pins as P
lib = oracle.load(SO)
# route every oracle call of the pins through the mutant
for name in ("validate", "eigenvalues", "sylvester", "std2", "swap", "reorder"):
    f = getattr(oracle, name)
    setattr(oracle, name, (lambda f: (lambda *a, **k: f(*a, lib=lib, **k)))(f))
checks = [
    lambda: [P.test_swap_1x1_closed_form(s) for s in range(3)],
    lambda: [P.test_std2_complex_closed_form(s) for s in range(3)],
    lambda: [P.test_std2_real_splits(s) for s in range(3)],
    lambda: [P.test_std2_real_nearly_triangular(M) for M in
             ([[2.0, 1.0], [1e-9, 1.0]], [[1.0, 3.0], [2e-12, -1.0]])],
    lambda: [P.test_sylvester_exact(pq, s) for pq in [(1, 2), (2, 1), (2, 2)] for s in range(2)],
    lambda: [P.test_swap_block_exact_subspace(pq, s) for pq in [(1, 2), (2, 1), (2, 2)] for s in range(3)],
    lambda: [P.test_bruteforce_all_selections(n) for n in (4, 6)],
    lambda: P.test_dtrsen_crosscheck(50, 2, 0.3),
    lambda: P.test_swap_decision_matches_dtrsen(),
    lambda: P.test_invariants_n400("n400"),
    lambda: P.test_edge_cases(),
    lambda: P.test_rejection_semantics(),
]
failed = 0
for c in checks:
    try:
        c()
    except Exception:
        failed += 1
print("FAILED_CHECKS", failed)
sys.exit(1 if failed else 0)
"""


def run_battery(so):
    code = BATTERY.replace("ROOT", repr(ROOT)).replace("SO", repr(so))
    try:
        p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=300, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return 124, "timeout"
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def src():
    with open(os.path.join(ROOT, "oracle", "reorder_oracle.c")) as f:
        return f.read()


def test_battery_passes_on_oracle(tmp_path):
    so = oracle.build(force=True, out=str(tmp_path / "orig.so"))
    rc, out = run_battery(so)
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_killed(src, name, old, new, tmp_path):
    assert old in src, f"mutation anchor for {name!r} not found"
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = oracle.build(force=True, src=str(c), out=str(tmp_path / "mut.so"))
    rc, out = run_battery(so)
    assert rc != 0, f"mutant {name!r} survived the pins"
