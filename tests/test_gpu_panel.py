"""One off-diagonal update Y <- Y U on one panel (Section 3.2, the level-3
step of a window) through gbr_update_panel, in both precisions.

FP64 DMMA and FP64 FMA tiles: against the exact product (long double
accumulation) within the forward error bound of a w-term dot product; the
FMA tile also bitwise against its stated operation order (one fused
multiply-add chain per output over k in increasing order, from +0),
emulated with exact rationals and one correct rounding per step.

Split precision (tcgen05): bitwise against an independent emulation of the
stated digit scheme, written here from its definition with numpy integer
matrix products and Python integers (55-bit fixed point relative to the
largest exponent of the row of Y / column of U, 7 balanced base-256 digits,
the slice products with p + q <= 8 summed exactly, one rounding to double),
and against the exact product within the stated bound
(2^-50 |y|max |u|max per term).
"""
import math
from fractions import Fraction

import numpy as np
import pytest


torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def _expo(x):
    return ((x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)


def _digits(x, emax):
    """The 7 balanced digits (p = 1..7) of every entry of x relative to the
    exponent field emax (broadcast against x): int64 array (7,) + x.shape."""
    b = x.view(np.uint64)
    e = _expo(x)
    m = (b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    sh = emax - e
    valid = (e != 0) & (sh < 64)
    shc = np.clip(sh, 0, 63).astype(np.uint64)
    F = np.where(valid, (m << np.uint64(2)) >> shc, np.uint64(0)).astype(np.int64)
    V = np.where((b >> np.uint64(63)) == 1, -F, F)
    G = V + 0x808080808080
    d = [G >> 48] + [((G >> (8 * (7 - p))) & 255) - 128 for p in range(2, 8)]
    return np.stack(d)


def emulate(Y, U):
    """Y U in the split-precision scheme, computed exactly and rounded once."""
    rows, w = Y.shape
    er = _expo(Y).max(axis=1) if w else np.zeros(rows, np.int64)
    ec = _expo(U).max(axis=0)
    Yd = _digits(Y, er[:, None])
    Ud = _digits(U, ec[None, :])
    D = {}
    for p in range(1, 8):
        for q in range(1, 9 - p):
            D[p + q] = D.get(p + q, 0) + Yd[p - 1] @ Ud[q - 1]
    T = np.zeros((rows, w), dtype=object)
    for d in range(2, 9):
        T = T * 256 + D[d].astype(object)
    out = np.zeros((rows, w))
    for r in range(rows):
        for n in range(w):
            if er[r] == 0 or ec[n] == 0:
                continue
            out[r, n] = math.ldexp(float(T[r, n]), -64 + int(er[r]) - 1021 + int(ec[n]) - 1021)
    return out


def exact(Y, U):
    return (Y.astype(np.longdouble) @ U.astype(np.longdouble)).astype(np.float64)


def make_case(rows, w, seed, extreme=False):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((rows, w))
    Y[::7] *= 2.0 ** rng.integers(-20, 21, size=(len(Y[::7]), 1))   # row scales
    Y[rng.random((rows, w)) < 0.05] = 0.0
    Y[::11, : w // 3] *= 2.0 ** -30                                   # spread inside a row
    U = rng.standard_normal((w, w)) / np.sqrt(w)
    k, n = np.indices((w, w))
    U[k > n + w // 3] = 0.0                                           # staircase of a window's U
    if extreme:
        # the entry whose 7 digits are all at the top of their range: the
        # diagonal sums reach the largest magnitudes the scheme allows
        xa = np.array([0x3FF0000000000000 | (0x1FDFDFDFDFDFDF & ((1 << 52) - 1))],
                      dtype=np.uint64).view(np.float64)[0]
        Y[::3] = xa
        U[:, ::2] = xa
    return Y, U


def to_panel(Y, layout):
    """Y as a CUDA tensor: 'col' column-major with ld = rows + 3 (rs = 1),
    'row' row-major with ld = w + 5 (ks = 1)."""
    rows, w = Y.shape
    if layout == "col":
        buf = torch.zeros((w, rows + 3), dtype=torch.float64, device="cuda")
        t = buf.t()[:rows]
    else:
        buf = torch.zeros((rows, w + 5), dtype=torch.float64, device="cuda")
        t = buf[:, :w]
    t.copy_(torch.from_numpy(Y))
    return t


def to_u(U):
    t = torch.empty((U.shape[1], U.shape[0] + 2), dtype=torch.float64, device="cuda").t()
    t = t[: U.shape[0]]
    t.copy_(torch.from_numpy(U))
    return t


CASES = [(1, 128, "col"), (300, 128, "col"), (300, 128, "row"), (257, 100, "row"),
         (77, 37, "col"), (129, 64, "row"), (200, 128, "col")]


@pytest.mark.parametrize("rows,w,layout", CASES)
def test_dmma_panel_against_exact(gbr, rows, w, layout):
    Y, U = make_case(rows, w, seed=rows * 1000 + w)
    t = to_panel(Y, layout)
    gbr.update_panel(t, to_u(U), "dmma")
    got = t.cpu().numpy()
    ref = exact(Y, U)
    bound = 2 * w * EPS * (np.abs(Y) @ np.abs(U))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


@pytest.mark.parametrize("rows,w,layout", CASES)
def test_fma_panel_against_exact(gbr, rows, w, layout):
    Y, U = make_case(rows, w, seed=rows * 1000 + w + 2)
    t = to_panel(Y, layout)
    gbr.update_panel(t, to_u(U), "fma")
    got = t.cpu().numpy()
    ref = exact(Y, U)
    bound = 2 * w * EPS * (np.abs(Y) @ np.abs(U))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


def fma_chain(Y, U):
    """Each output as acc = fma(y_k, u_k, acc) over k = 0..w-1 from +0, every
    step rounded once (Python's int/int division rounds correctly)."""
    rows, w = Y.shape
    out = np.zeros((rows, w))
    for r in range(rows):
        for n in range(w):
            acc = 0.0
            for k in range(w):
                if U[k, n] == 0.0 or Y[r, k] == 0.0:
                    continue      # fma(y, 0, acc) = acc exactly (finite y, acc)
                exact_v = Fraction(Y[r, k]) * Fraction(U[k, n]) + Fraction(acc)
                acc = exact_v.numerator / exact_v.denominator if exact_v != 0 else 0.0
            out[r, n] = acc
    return out


@pytest.mark.parametrize("rows,w,layout", [(70, 24, "col"), (33, 19, "row")])
def test_fma_panel_bitwise_chain(gbr, rows, w, layout):
    Y, U = make_case(rows, w, seed=rows + w)
    t = to_panel(Y, layout)
    gbr.update_panel(t, to_u(U), "fma")
    got = t.cpu().numpy()
    want = fma_chain(Y, U)
    mism = np.argwhere(got.view(np.uint64) != want.view(np.uint64))
    assert mism.size == 0, f"{len(mism)} outputs differ, first {mism[:3].tolist()}"


@pytest.mark.parametrize("rows,w,layout", CASES)
def test_split_precision_panel_bitwise(gbr, rows, w, layout):
    extreme = (rows, w) == (200, 128)
    Y, U = make_case(rows, w, seed=rows * 1000 + w + 1, extreme=extreme)
    t = to_panel(Y, layout)
    gbr.update_panel(t, to_u(U), "ozaki")
    got = t.cpu().numpy()
    want = emulate(Y, U)
    mism = np.argwhere(got.view(np.uint64) != want.view(np.uint64))
    assert mism.size == 0, f"{len(mism)} outputs differ, first {mism[:3].tolist()}"
    # the stated error bound against the exact product
    ym = np.abs(Y).max(axis=1)[:, None]
    um = np.abs(U).max(axis=0)[None, :]
    assert np.all(np.abs(got - exact(Y, U)) <= w * 2.0 ** -50 * ym * um + 1e-300)


def test_panel_calls_in_a_row_and_zero_rows(gbr):
    """Consecutive calls with different U reuse the library's scratch; a
    0-row panel is a no-op."""
    for s in range(2):
        Y, U = make_case(150, 96, seed=50 + s)
        t = to_panel(Y, "col")
        gbr.update_panel(t, to_u(U), "ozaki")
        assert np.array_equal(t.cpu().numpy().view(np.uint64), emulate(Y, U).view(np.uint64))
    e = torch.zeros((0, 16), dtype=torch.float64, device="cuda")
    gbr.update_panel(e, to_u(np.eye(16)), "ozaki")
