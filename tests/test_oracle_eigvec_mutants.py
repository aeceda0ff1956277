"""The eigenvector oracle's pins must catch plausible mistakes.

Each case plants one mistake (a wrong sign, a transposed operand, a dropped
block, a disabled overflow guard, a wrong norm) in a temporary copy of
`oracle/eigvec_oracle.c`, compiles it with the unmodified reordering source,
and runs the pins of tests/test_oracle_eigvec.py against it in a subprocess.
The battery must fail for every mutant and pass for the unmodified source.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EV_SRC = os.path.join(ROOT, "oracle", "eigvec_oracle.c")
RE_SRC = os.path.join(ROOT, "oracle", "reorder_oracle.c")

MUTANTS = [
    ("start vector of a pair", "y[j + 1].im = w / b;", "y[j + 1].im = -w / b;"),
    ("right-hand side sign", "s.re -= AT(S, ldS, i, t) * y[t].re;", "s.re += AT(S, ldS, i, t) * y[t].re;"),
    ("update transposed", "r[i].re -= AT(S, ldS, i, b0 + t) * x[t].re;",
     "r[i].re -= AT(S, ldS, b0 + t, i) * x[t].re;"),
    ("2x2 block above taken as 1x1",
     "const int b0 = (b1 >= 2 && AT(S, ldS, b1 - 1, b1 - 2) != 0.0) ? b1 - 2 : b1 - 1;",
     "const int b0 = b1 - 1;"),
    ("adjugate entry", "cplx u1 = csub(cmul(m00, r[b0 + 1]), cmul(m10, r[b0]));",
     "cplx u1 = csub(cmul(m00, r[b0 + 1]), cmul(m01, r[b0]));"),
    ("no scaling before a division",
     "for (int it = 0; it < 8 && cabs1(r[b0]) > BIG * cabs1(d); ++it) {",
     "for (int it = 0; it < 0 && cabs1(r[b0]) > BIG * cabs1(d); ++it) {"),
    ("no scaling before an update", "for (int it = 0; it < 8 && rb + k * cm * xm > BIG; ++it) {",
     "for (int it = 0; it < 0 && rb + k * cm * xm > BIG; ++it) {"),
    ("pair selected by its first row only",
     "int sel = select ? (select[j] != 0 || (nb == 2 && select[j + 1] != 0)) : 1;",
     "int sel = select ? (select[j] != 0) : 1;"),
    ("real and imaginary columns exchanged",
     "for (int i = 0; i < n; ++i) AT(Y, ldY, i, m) = y[i].re;",
     "for (int i = 0; i < n; ++i) AT(Y, ldY, i, m) = nb == 2 ? y[i].im : y[i].re;"),
    ("normalization norm", "for (int i = 0; i < top; ++i) mx = fmax(mx, cabs1(y[i]));",
     "for (int i = 0; i < top; ++i) mx = fmax(mx, fabs(y[i].re));"),
]

BATTERY = r"""
import sys, numpy as np
sys.path.insert(0, ROOT)
import oracle
from tests import test_oracle_eigvec as P
lib = oracle.load(SO)
f = oracle.eigenvectors
oracle.eigenvectors = lambda *a, **k: f(*a, lib=lib, **k)
checks = [
    lambda: [P.test_residual_and_normalization(n, s) for n, s in [(7, 2), (60, 3)]],
    lambda: P.test_against_lapack_geev(),
    lambda: P.test_two_by_two_block_closed_form(),
    lambda: P.test_overflow_protection_against_exact_rationals(),
    lambda: P.test_each_overflow_guard_is_needed("tiny pivots"),
    lambda: P.test_each_overflow_guard_is_needed("huge couplings"),
    lambda: P.test_selection_and_repeated_eigenvalue(),
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


def build(ev_src, out):
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-o", out,
           RE_SRC, ev_src, "-lm"]
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
    so = build(EV_SRC, str(tmp_path / "orig.so"))
    rc, out = run_battery(so)
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_killed(name, old, new, tmp_path):
    with open(EV_SRC) as f:
        src = f.read()
    assert old in src, f"mutation anchor for {name!r} not found"
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new, 1))
    so = build(str(c), str(tmp_path / "mut.so"))
    rc, out = run_battery(so)
    assert rc != 0, f"mutant {name!r} survived the pins"
