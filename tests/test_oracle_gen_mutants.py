"""The generalized reordering oracle's pins must catch plausible mistakes.

Each case plants one mistake (a wrong sign, a transposed operand, a factor
taken from the wrong solution, a dropped step) in a temporary copy of
`oracle/gen_oracle.c`, compiles it with the unmodified standard-form
sources, and runs the pins of tests/test_oracle_gen.py against it in a
subprocess.  The battery must fail for every mutant and pass for the
unmodified source.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN_SRC = os.path.join(ROOT, "oracle", "gen_oracle.c")
OTHER = [os.path.join(ROOT, "oracle", "reorder_oracle.c"), os.path.join(ROOT, "oracle", "eigvec_oracle.c")]

MUTANTS = [
    ("right-hand side sign", "b[row] = -D[(p + c) * 4 + i];", "b[row] = D[(p + c) * 4 + i];"),
    ("sign of the L term", "K[row][pq + i + p * m] -= D[(p + c) * 4 + p + m];",
     "K[row][pq + i + p * m] += D[(p + c) * 4 + p + m];"),
    ("A22 transposed", "K[row][pq + i + p * m] -= D[(p + c) * 4 + p + m];",
     "K[row][pq + i + p * m] -= D[(p + m) * 4 + p + c];"),
    ("Q from the right solution", "qr_factor(p, q, L, gamma, Qs);", "qr_factor(p, q, R, gamma, Qs);"),
    ("rows updated by Qs, not Qs^T", "s += Qs[r * 4 + t] * EL(A, ld, j + t, c);",
     "s += Qs[t * 4 + r] * EL(A, ld, j + t, c);"),
    ("columns updated by Zs^T", "s += EL(A, ld, r, j + t) * Zs[c * 4 + t];",
     "s += EL(A, ld, r, j + t) * Zs[t * 4 + c];"),
    ("Q and Z factors exchanged", "const double *F = e ? Zs : Qs;", "const double *F = e ? Qs : Zs;"),
    ("T block not triangularized", "if (sz != 2) continue;", "if (sz != 2 || 1) continue;"),
    ("rotation sign", "double c = b11 / h, s = -b10 / h;", "double c = b11 / h, s = b10 / h;"),
    ("eigenvalue real part", "double re = b / (2.0 * a), im", "double re = b / a, im"),
    ("pencil coefficient sign", "*b = s11 * t22 + s22 * t11 - s21 * t12;",
     "*b = s11 * t22 + s22 * t11 + s21 * t12;"),
    ("second reflector skipped", "house0(k - 1, x, v2, &tau2);", "tau2 = 0.0;"),
    ("weak test dropped", "if (lowa > tha || lowb > thb) return 1;", ";"),
    ("old flags kept at the moved block", "for (int i = j + q; i < j + q + pa; ++i) sel[i] = 0;",
     "for (int i = j + q; i < j + q; ++i) sel[i] = 0;"),
    ("block above taken as 1x1",
     "const int pa = (here - 2 >= ks && EL(S, ldS, here - 1, here - 2) != 0.0) ? 2 : 1;",
     "const int pa = 1;"),
    ("2x2 selection not merged", "sel[j] = sel[j + 1] = s2;", "(void)s2;"),
    ("real pair roots swapped", "wr[j] = m + r; wi[j] = 0.0;\n                wr[j + 1] = m - r;",
     "wr[j] = m - r; wi[j] = 0.0;\n                wr[j + 1] = m + r;"),
]

BATTERY = r"""
import sys, numpy as np
sys.path.insert(0, ROOT)
import oracle
oracle._lib = oracle.load(SO)
from tests import test_oracle_gen as P
checks = [
    lambda: [P.test_invariants_and_order(n, s) for n, s in [(3, 2), (12, 4), (60, 5)]],
    lambda: P.test_against_lapack_ordqz(),
    lambda: P.test_generalized_eigenvalues_against_lapack(),
    lambda: P.test_reduces_to_standard_reordering(),
    lambda: P.test_two_1x1_blocks_closed_form(),
    lambda: [P.test_local_swap_every_type(p, q) for p, q in [(1, 1), (1, 2), (2, 1), (2, 2)]],
    lambda: [P.test_generalized_sylvester_residual(p, q) for p, q in [(1, 1), (1, 2), (2, 1), (2, 2)]],
    lambda: P.test_equal_eigenvalues_and_selection_rules(),
    lambda: P.test_rejected_swap_changes_nothing(),
    lambda: P.test_eigenvalues_of_a_real_pair_block(),
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


def build(gen_src, out):
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-o", out,
           *OTHER, gen_src, "-lm"]
    subprocess.run(cmd, check=True)
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
    so = build(GEN_SRC, str(tmp_path / "orig.so"))
    rc, out = run_battery(so)
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_killed(name, old, new, tmp_path):
    with open(GEN_SRC) as f:
        src = f.read()
    assert old in src, f"mutation anchor for {name!r} not found"
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = build(str(c), str(tmp_path / "mut.so"))
    rc, out = run_battery(so)
    assert rc != 0, f"mutant {name!r} survived the pins"
