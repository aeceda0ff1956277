"""Pins of the eigenvector oracle (Eq. 5: (S - lambda I) y = 0, back-transform
x = Q y of Eq. 6, overflow protection): closed forms, exact rational
arithmetic, an independent library (numpy/LAPACK geev), invariants."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import schur_inputs as si

EPS = np.finfo(np.float64).eps


def complex_columns(X, kinds, lams):
    """(vector, eigenvalue) per eigenvector, complex vectors from their pair."""
    out, c = [], 0
    while c < X.shape[1]:
        if kinds[c] == 0:
            out.append((X[:, c].astype(complex), lams[c]))
            c += 1
        else:
            out.append((X[:, c] + 1j * X[:, c + 1], lams[c]))
            c += 2
    return out


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (60, 3), (200, 4)])
def test_residual_and_normalization(n, seed):
    S, Q, _ = si.reorder_problem(n, seed, select_frac=0.5, q="householder", reflectors=8)
    X, kinds, lams, ns = oracle.eigenvectors(S)
    assert X.shape == (n, n) and np.all(ns == 0)
    for y, lam in complex_columns(X, kinds, lams):
        assert np.linalg.norm(S @ y - lam * y) <= 10 * n * EPS * np.linalg.norm(S) * np.linalg.norm(y)
        # normalization: max |re| + |im| = 1
        assert abs(np.max(np.abs(y.real) + np.abs(y.imag)) - 1.0) <= 4 * EPS
    # back-transformed: A x = lambda x with A = Q S Q^T
    A = Q @ S @ Q.T
    Xb, kinds, lams, _ = oracle.eigenvectors(S, Q)
    for x, lam in complex_columns(Xb, kinds, lams):
        assert np.linalg.norm(A @ x - lam * x) <= 20 * n * EPS * np.linalg.norm(A) * np.linalg.norm(x)


def test_against_lapack_geev():
    """Each eigenvector is parallel to the one numpy (LAPACK geev) computes
    from A = Q S Q^T.  The coupling above the diagonal blocks is scaled down
    so that every eigenvalue is well conditioned."""
    n = 40
    S, Q, _ = si.reorder_problem(n, 11, select_frac=0.5, q="householder", reflectors=8)
    in_block = np.zeros((n, n), dtype=bool)
    for j in range(n - 1):
        if S[j + 1, j] != 0.0:
            in_block[j, j + 1] = True
    S[np.triu(np.ones((n, n), dtype=bool), 1) & ~in_block] *= 0.05
    A = Q @ S @ Q.T
    w, V = np.linalg.eig(A)
    X, kinds, lams, _ = oracle.eigenvectors(S, Q)
    for x, lam in complex_columns(X, kinds, lams):
        i = int(np.argmin(np.abs(w - lam)))
        gap = np.sort(np.abs(w - lam))[1]
        assert abs(w[i] - lam) <= 1e-10 * max(1.0, abs(lam))
        cos = abs(np.vdot(V[:, i], x)) / (np.linalg.norm(V[:, i]) * np.linalg.norm(x))
        assert 1.0 - cos <= 1e-20 / gap ** 2 + 1e-12


def test_two_by_two_block_closed_form():
    """For the standardized block [[a, b], [c, a]] the vector of
    lambda = a + i sqrt(-bc) is (1, i sqrt(-bc) / b), normalized."""
    a, b, c = 0.75, 1.5, -0.5
    S = np.array([[a, b], [c, a]])
    X, kinds, lams, _ = oracle.eigenvectors(S)
    w = np.sqrt(-b * c)
    assert list(kinds) == [1, 2] and lams[0] == complex(a, w)
    v = np.array([1.0, 1j * w / b])
    v /= np.max(np.abs(v.real) + np.abs(v.imag))
    assert np.allclose(X[:, 0] + 1j * X[:, 1], v, rtol=0, atol=4 * EPS)


def exact_triangular_eigvec(T, j):
    """Eigenvector of the upper triangular T (exact binary fractions) for the
    eigenvalue T[j, j], by exact rational back substitution, normalized."""
    n = T.shape[0]
    F = [[Fraction(float(T[i, k])) for k in range(n)] for i in range(n)]
    lam = F[j][j]
    y = [Fraction(0)] * n
    y[j] = Fraction(1)
    for i in range(j - 1, -1, -1):
        s = sum(F[i][k] * y[k] for k in range(i + 1, j + 1))
        y[i] = -s / (F[i][i] - lam)
    m = max(abs(v) for v in y)
    return np.array([float(v / m) for v in y])


def test_overflow_protection_against_exact_rationals():
    """Tiny eigenvalue gaps with large couplings: the unscaled vector grows
    by 2^60 per row and would overflow after ~17 rows.  The oracle rescales
    (by exact powers of two) and matches exact rational back substitution."""
    n = 40
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = 1.0 + i * 2.0 ** -30
        T[i, i + 1:] = 2.0 ** 30 * (1 + (np.arange(i + 1, n) % 3))
    X, kinds, lams, ns = oracle.eigenvectors(T)
    assert np.all(np.isfinite(X))
    assert ns[n - 1] > 0  # the last vector needed scaling
    for j in (n - 1, n // 2, 3):
        want = exact_triangular_eigvec(T, j)
        assert np.allclose(X[:, j], want, rtol=1e-12, atol=1e-300)


def test_selection_and_repeated_eigenvalue():
    """Selected columns are the corresponding columns of the full set; a
    repeated eigenvalue (zero pivot) is perturbed to smin and stays finite."""
    n = 30
    S, _, _ = si.reorder_problem(n, 5, select_frac=0.5, q="identity")
    Xall, kinds, _, _ = oracle.eigenvectors(S)
    sel = np.zeros(n, dtype=np.int32)
    sel[::3] = 1
    Xs, ksel, _, _ = oracle.eigenvectors(S, select=sel)
    # map selected positions to columns of the full result
    cols, c, j = [], 0, 0
    while j < n:
        nb = 2 if (j + 1 < n and S[j + 1, j] != 0) else 1
        if sel[j] or (nb == 2 and sel[j + 1]):
            cols += list(range(c, c + nb))
        c += nb
        j += nb
    assert np.array_equal(Xs, Xall[:, cols])
    T = np.array([[1.0, 1.0], [0.0, 1.0]])
    X, _, _, _ = oracle.eigenvectors(T)
    assert np.all(np.isfinite(X))
    assert abs(X[0, 1]) == 1.0 and abs(X[1, 1]) < 1e-14  # direction e1 (defective)


@pytest.mark.parametrize("kind", ["tiny pivots", "huge couplings"])
def test_each_overflow_guard_is_needed(kind):
    """Two growth patterns, each stopped by a different guard:
    eigenvalues near 0 with gaps of 2^-600 (a division by a tiny pivot
    overflows unless the vector is scaled first), and couplings of 2^300 (an
    update overflows unless scaled first).  Compared with exact rational
    back substitution."""
    n = 12
    T = np.zeros((n, n))
    for i in range(n):
        if kind == "tiny pivots":
            T[i, i] = i * 2.0 ** -600
            T[i, i + 1:] = 1.0 + (np.arange(i + 1, n) % 2)
        else:
            T[i, i] = 1.0 + i
            T[i, i + 1:] = 2.0 ** 300 * (1 + (np.arange(i + 1, n) % 3))
    X, _, _, ns = oracle.eigenvectors(T)
    assert np.all(np.isfinite(X))
    assert ns[n - 1] > 0
    for j in (n - 1, n - 3):
        want = exact_triangular_eigvec(T, j)
        assert np.allclose(X[:, j], want, rtol=1e-12, atol=1e-300)
