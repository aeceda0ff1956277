"""Pins of the bulge-chasing sweep oracle (Section 3.2: one pipelined QR
iteration by overlapping 3x3 Householder reflectors on an upper Hessenberg
matrix): the implicit-Q theorem against an explicit QR factorization of the
shift polynomial (numpy/LAPACK), deflation with exact shifts, invariants."""
import numpy as np
import pytest

import oracle
import schur_inputs as si

EPS = np.finfo(np.float64).eps


def shift_polynomial(H, shifts):
    """p(H) = prod over pairs of (H^2 - s H + p I)."""
    n = H.shape[0]
    M = np.eye(n)
    for b in range(len(shifts) // 2):
        s = (shifts[2 * b] + shifts[2 * b + 1]).real
        p = (shifts[2 * b] * shifts[2 * b + 1]).real
        M = (H @ H - s * H + p * np.eye(n)) @ M
    return M


@pytest.mark.parametrize("n,ns,tol", [(5, 2, 1e-14), (12, 2, 1e-14), (40, 2, 1e-13),
                                      (12, 4, 1e-13), (20, 6, 1e-13), (30, 8, 1e-11)])
def test_implicit_q_theorem(n, ns, tol):
    """The swept H equals Qe^T H Qe for the orthogonal factor Qe of
    p(H) = Qe R (explicit QR through numpy): both are unreduced Hessenberg
    matrices whose orthogonal factor has the first column of p(H) e_1, so
    they agree up to the signs of the columns (compared as magnitudes)."""
    H, _, sh = si.hessenberg_problem(n, 100 + n + ns, nshifts=ns, reflectors=4)
    st, H2, _ = oracle.qr_sweep(H, None, sh)
    assert st == 0
    Qe, _ = np.linalg.qr(shift_polynomial(H, sh))
    He = Qe.T @ H @ Qe
    assert np.max(np.abs(np.abs(He) - np.abs(H2))) <= tol * np.linalg.norm(H)


@pytest.mark.parametrize("n,ns", [(3, 2), (4, 2), (9, 4), (60, 8), (200, 16)])
def test_invariants(n, ns):
    """Upper Hessenberg with exact zeros below the subdiagonal, Q orthogonal,
    and Q H Q^T unchanged (backward error at rounding level)."""
    H, Q, sh = si.hessenberg_problem(n, n, nshifts=ns, reflectors=8)
    A = Q @ H @ Q.T
    st, H2, Q2 = oracle.qr_sweep(H, Q, sh)
    assert st == 0
    assert np.all(np.tril(H2, -2) == 0.0)
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(n)) <= 20 * n * EPS
    assert np.linalg.norm(A - Q2 @ H2 @ Q2.T) <= 20 * n * EPS * np.linalg.norm(A)
    ev0 = np.sort_complex(np.linalg.eigvals(H))
    ev1 = np.sort_complex(np.linalg.eigvals(H2))
    assert np.max(np.abs(ev0 - ev1)) <= 1e-8 * max(1.0, np.max(np.abs(ev0)))


def test_exact_shifts_deflate():
    """A sweep whose shifts are a conjugate pair of eigenvalues of H splits
    off that pair at the bottom (H[n-2, n-3] vanishes); two real
    eigenvalues as shifts deflate the last one (H[n-1, n-2])."""
    n = 30
    H, _, _ = si.hessenberg_problem(n, 3, nshifts=2, reflectors=4)
    w = np.linalg.eigvals(H)
    c = [x for x in w if x.imag > 1e-3][0]
    st, H2, _ = oracle.qr_sweep(H, None, [c, np.conj(c)])
    assert st == 0 and abs(H2[n - 2, n - 3]) <= 1e-10 * np.linalg.norm(H)
    assert abs(H[n - 2, n - 3]) > 1e-3
    r = [x for x in w if abs(x.imag) < 1e-12][:2]
    st, H3, _ = oracle.qr_sweep(H, None, r)
    assert st == 0 and abs(H3[n - 1, n - 2]) <= 1e-10 * np.linalg.norm(H)


def test_two_by_two_pair_closed_form():
    """n = 3, one bulge: the sweep is a single reflector on rows/columns 0..2
    from x = (H^2 - s H + p I) e_1 and one 2x2 reflector; the result's first
    column of Q spans x (the Francis step's defining vector)."""
    H = np.array([[1.0, 2.0, 0.5], [0.7, -1.0, 1.5], [0.0, 0.4, 2.0]])
    sh = [complex(0.3, 0.8), complex(0.3, -0.8)]
    st, H2, Q2 = oracle.qr_sweep(H, np.eye(3), sh)
    assert st == 0
    x = shift_polynomial(H, sh)[:, 0]
    q0 = Q2[:, 0]
    assert abs(abs(q0 @ x) / np.linalg.norm(x) - 1.0) <= 8 * EPS
    assert H2[2, 0] == 0.0


def test_argument_checks():
    H, _, _ = si.hessenberg_problem(6, 1, nshifts=2)
    assert oracle.qr_sweep(H, None, [1.0, 2.0, 3.0])[0] == -1          # odd count
    assert oracle.qr_sweep(H, None, [complex(1, 1), complex(2, -1)])[0] == -1  # not a pair
    Hb = H.copy()
    Hb[4, 1] = 1.0
    assert oracle.qr_sweep(Hb, None, [1.0, 2.0])[0] == -2               # not Hessenberg
    st, H1, _ = oracle.qr_sweep(H, None, [])
    assert st == 0 and np.array_equal(H1, H)
