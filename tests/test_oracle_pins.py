"""Pins of the CPU oracle against what the mathematics fixes.

The paper (Section 2, Eq. 7; Section 3.2) defines the result -- an
orthogonal similarity that moves the selected eigenvalues of a real Schur
form to its leading diagonal blocks -- but prints no worked example.  The
oracle is therefore pinned to things other than itself:

* closed forms (1x1 swap, 2x2 standardization);
* exact rational solutions of the small Sylvester equations (sympy, from
  the defining equation T11 X - X T22 = T12) and the exactly known swapped
  subspace span([-X; I]);
* brute force on tiny inputs: every selection, compared with the invariant
  subspace spanned by numpy eigenvectors of the selected eigenvalues;
* an independent library: LAPACK dtrsen through scipy (called, not read);
* invariants at any size.
"""
import itertools

import numpy as np
import pytest
import sympy
from scipy.linalg import lapack
from scipy.optimize import linear_sum_assignment

import oracle
import schur_inputs as si
from tests.helpers import (EPS, block_eigs, blocks, expected_order, is_standard,
                           match_eigs, orth_err, residual, sin_angle)


def dtrsen_sep(S, select):
    n = S.shape[0]
    m = int(np.sum(select))
    lw = max(1, 2 * m * (n - m))
    out = lapack.dtrsen(np.asarray(select, dtype=np.int32), S, np.eye(n), job="V",
                        lwork=lw, liwork=max(1, m * (n - m)))
    return out[6]


def well_conditioned_schur(n, rng, upper_scale=0.05):
    """Schur form from the standard generator laws but with a small strict
    upper part, so that sep (and the subspace condition) is moderate."""
    S, sizes = si.schur_form(n, rng)
    mask = np.triu(np.ones((n, n), dtype=bool), 1)
    for j, sz in blocks(S):
        if sz == 2:
            mask[j, j + 1] = False
    S[mask] *= upper_scale
    return S, sizes


# ---------------------------------------------------------------- 1x1 swap

@pytest.mark.parametrize("seed", range(8))
def test_swap_1x1_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    n = 5
    S = np.triu(rng.standard_normal((n, n)))
    S = np.asfortranarray(S)
    j = 1
    t11, t12, t22 = S[j, j], S[j, j + 1], S[j + 1, j + 1]
    st, Sn, Qn = oracle.swap(S, j, 1, 1, Q=np.eye(n))
    assert st == 0
    # swapped diagonal, exactly; |t12| preserved
    assert Sn[j, j] == t22 and Sn[j + 1, j + 1] == t11
    assert Sn[j + 1, j] == 0.0
    assert abs(abs(Sn[j, j + 1]) - abs(t12)) <= 8 * EPS * abs(t12)
    # the transformation is a plane rotation in (j, j+1) whose first column
    # is the eigenvector (t12, t22 - t11) of t22
    G = Qn[j:j + 2, j:j + 2]
    assert np.allclose(np.delete(np.delete(Qn, [j, j + 1], 0), [j, j + 1], 1), np.eye(n - 2))
    assert abs(np.linalg.det(G) - 1.0) < 1e-14
    v = np.array([t12, t22 - t11])
    v /= np.linalg.norm(v)
    assert abs(abs(G[:, 0] @ v) - 1.0) < 1e-14
    # it is a similarity: Q^T S Q = S_new
    assert np.linalg.norm(Qn.T @ S @ Qn - Sn) <= 20 * EPS * np.linalg.norm(S)
    assert orth_err(Qn) <= 10 * EPS


# --------------------------------------------------- 2x2 standardization

@pytest.mark.parametrize("seed", range(10))
def test_std2_complex_closed_form(seed):
    rng = np.random.default_rng(200 + seed)
    while True:
        M = rng.standard_normal((2, 2))
        tr, det = np.trace(M), np.linalg.det(M)
        if tr * tr - 4 * det < -0.1:   # complex pair
            break
    c, s, N = oracle.std2(M)
    Z = np.array([[c, -s], [s, c]])
    assert abs(c * c + s * s - 1) < 4 * EPS
    assert N[0, 0] == N[1, 1]
    assert N[0, 1] * N[1, 0] < 0
    assert abs(np.trace(N) - tr) < 1e-14 * (1 + abs(tr))
    assert abs(np.linalg.det(N) - det) < 1e-14 * (1 + abs(det))
    assert np.linalg.norm(Z.T @ M @ Z - N) < 8 * EPS * np.linalg.norm(M)
    # the standardized block's eigenvalues a +- i sqrt(-bc) are M's
    ev = np.sort_complex(np.linalg.eigvals(M))
    a, im = N[0, 0], np.sqrt(-N[0, 1] * N[1, 0])
    assert np.allclose(np.sort_complex(np.array([a - 1j * im, a + 1j * im])), ev, rtol=1e-13)


@pytest.mark.parametrize("seed", range(10))
def test_std2_real_splits(seed):
    rng = np.random.default_rng(300 + seed)
    while True:
        M = rng.standard_normal((2, 2))
        tr, det = np.trace(M), np.linalg.det(M)
        if tr * tr - 4 * det > 0.1 and M[1, 0] != 0:
            break
    c, s, N = oracle.std2(M)
    Z = np.array([[c, -s], [s, c]])
    assert N[1, 0] == 0.0
    assert np.linalg.norm(Z.T @ M @ Z - N) < 8 * EPS * np.linalg.norm(M)
    roots = np.sort(np.roots([1.0, -tr, det]).real)
    assert np.allclose(np.sort([N[0, 0], N[1, 1]]), roots, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("M", [[[2.0, 1.0], [1e-9, 1.0]], [[1.0, 3.0], [2e-12, -1.0]],
                               [[-1.0, 1e-8], [4.0, 2.0]], [[0.5, -2.0], [-1e-11, 0.25]]])
def test_std2_real_nearly_triangular(M):
    """Real pair with |m12 m21| << ((m11 - m22)/2)^2: the Schur vector must
    be formed without cancellation, so that the forced zero below the
    diagonal is a backward error of order eps."""
    M = np.array(M)
    c, s, N = oracle.std2(M)
    Z = np.array([[c, -s], [s, c]])
    assert N[1, 0] == 0.0
    assert np.linalg.norm(Z.T @ M @ Z - N) < 8 * EPS * np.linalg.norm(M)


def test_std2_special_cases():
    # already triangular: identity rotation, block unchanged
    c, s, N = oracle.std2(np.array([[1.0, 2.0], [0.0, 3.0]]))
    assert (c, s) == (1.0, 0.0) and N[1, 0] == 0 and N[0, 0] == 1 and N[1, 1] == 3
    # zero (1,2) entry: a quarter turn makes it triangular
    c, s, N = oracle.std2(np.array([[1.0, 0.0], [5.0, 3.0]]))
    assert N[1, 0] == 0 and {N[0, 0], N[1, 1]} == {1.0, 3.0}
    # already standard: unchanged
    c, s, N = oracle.std2(np.array([[0.5, 2.0], [-1.0, 0.5]]))
    assert (c, s) == (1.0, 0.0) and np.array_equal(N, np.array([[0.5, 2.0], [-1.0, 0.5]]))


# ------------------------------------------------- Sylvester, exact rationals

def exact_sylvester(T11, T22, T12):
    """Exact X with T11 X - X T22 = T12, solved by sympy from the equation."""
    p, q = T11.shape[0], T22.shape[0]
    xs = sympy.symbols(f"x0:{p * q}")
    X = sympy.Matrix(p, q, xs)
    A, B, C = (sympy.Matrix(T11.astype(int).tolist()), sympy.Matrix(T22.astype(int).tolist()),
               sympy.Matrix(T12.astype(int).tolist()))
    sol = sympy.solve(list(A * X - X * B - C), xs, dict=True)[0]
    return np.array([[float(sol[X[i, k]]) for k in range(q)] for i in range(p)])


def int_std_block(rng):
    """Integer standardized 2x2 block [[a, b], [c, a]], bc < 0."""
    a = int(rng.integers(-4, 5))
    b = int(rng.integers(1, 5)) * int(rng.choice([-1, 1]))
    c = -int(np.sign(b)) * int(rng.integers(1, 5))
    return np.array([[a, b], [c, a]], dtype=float)


def int_case(p, q, rng):
    T11 = int_std_block(rng) if p == 2 else np.array([[float(rng.integers(-6, 7))]])
    T22 = int_std_block(rng) if q == 2 else np.array([[float(rng.integers(-6, 7))]])
    if p == 1 and q == 1:
        while T22[0, 0] == T11[0, 0]:
            T22 = np.array([[float(rng.integers(-6, 7))]])
    if p == 2 and q == 2:
        while T22[0, 0] == T11[0, 0]:
            T22 = int_std_block(rng)
    T12 = rng.integers(-5, 6, (p, q)).astype(float)
    return T11, T22, T12


@pytest.mark.parametrize("pq", [(1, 2), (2, 1), (2, 2), (1, 1)])
@pytest.mark.parametrize("seed", range(6))
def test_sylvester_exact(pq, seed):
    p, q = pq
    rng = np.random.default_rng(400 + 10 * seed + p * 3 + q)
    T11, T22, T12 = int_case(p, q, rng)
    X, g = oracle.sylvester(T11, T22, T12)
    Xe = exact_sylvester(T11, T22, T12)
    assert 0 < g <= 1.0
    assert np.allclose(X / g, Xe, rtol=1e-13, atol=1e-13 * (1 + np.abs(Xe).max()))


@pytest.mark.parametrize("pq", [(1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("seed", range(8))
def test_swap_block_exact_subspace(pq, seed):
    """After the swap, the leading q columns of the accumulated Q span the
    exact invariant subspace span([-X; I]) of T22's eigenvalues, and the two
    new blocks carry T22's and T11's eigenvalues (closed forms)."""
    p, q = pq
    rng = np.random.default_rng(500 + 10 * seed + p * 3 + q)
    T11, T22, T12 = int_case(p, q, rng)
    k = p + q
    D = np.zeros((k, k))
    D[:p, :p], D[p:, p:], D[:p, p:] = T11, T22, T12
    D = np.asfortranarray(D)
    assert oracle.validate(D) == 0
    st, Dn, Qn = oracle.swap(D, 0, p, q, Q=np.eye(k))
    assert st == 0
    assert is_standard(Dn)
    Xe = exact_sylvester(T11, T22, T12)
    V = np.vstack([-Xe, np.eye(q)])
    sep_lb = 1.0 / np.linalg.norm(np.linalg.pinv(np.kron(np.eye(q), T11) - np.kron(T22.T, np.eye(p))), 2)
    assert sin_angle(Qn[:, :q], V) <= 1e-14 * max(1.0, np.linalg.norm(D) / sep_lb)
    # eigenvalues moved as whole blocks
    ev_new = block_eigs(Dn)
    ev22 = block_eigs(T22)
    ev11 = block_eigs(T11)
    assert np.allclose(np.sort_complex(ev_new[:q]), np.sort_complex(ev22), atol=1e-13)
    assert np.allclose(np.sort_complex(ev_new[q:]), np.sort_complex(ev11), atol=1e-13)
    assert np.linalg.norm(Qn.T @ D @ Qn - Dn) <= 50 * EPS * np.linalg.norm(D)
    assert orth_err(Qn) <= 20 * EPS


def test_swap_equal_spectra_stays_valid():
    """Two blocks with identical eigenvalues: any outcome the stability test
    accepts must still be an orthogonal similarity in standard form."""
    T = np.array([[0.5, 1.0], [-2.0, 0.5]])
    D = np.zeros((4, 4))
    D[:2, :2] = T
    D[2:, 2:] = T
    D[:2, 2:] = np.array([[1.0, -3.0], [2.0, 0.7]])
    D = np.asfortranarray(D)
    st, Dn, Qn = oracle.swap(D, 0, 2, 2, Q=np.eye(4))
    if st == 0:
        assert is_standard(Dn)
        assert np.linalg.norm(Qn.T @ D @ Qn - Dn) <= 50 * EPS * np.linalg.norm(D)
    else:
        assert np.array_equal(Dn, D)


def hard_swap_case(rng):
    """Adjacent blocks with close eigenvalues and strongly non-normal 2x2
    blocks: the regime where the direct swap can be unstable."""
    while True:
        p, q = int(rng.integers(1, 3)), int(rng.integers(1, 3))
        if p + q > 2:
            break
    a = rng.standard_normal()
    kappa = 10 ** rng.uniform(0, 8)
    b, c = rng.uniform(0.1, 2) * kappa, -rng.uniform(0.1, 2) / kappa
    delta = 10 ** rng.uniform(-16, -2)

    def blk(sz, a0, b0, c0):
        return np.array([[a0]]) if sz == 1 else np.array([[a0, b0], [c0, a0]])
    T11 = blk(p, a, b, c)
    T22 = blk(q, a + delta * rng.standard_normal(), b * (1 + delta), c)
    T12 = rng.standard_normal((p, q)) * 10 ** rng.uniform(-3, 6)
    D = np.zeros((p + q, p + q))
    D[:p, :p], D[p:, p:], D[:p, p:] = T11, T22, T12
    return np.asfortranarray(D), p, q


def test_swap_decision_matches_dtrsen():
    """Accept/reject decisions of the weak+strong stability test agree with
    LAPACK's dtrsen (an independent implementation of the same test) on
    random hard swaps; both outcomes occur."""
    rng = np.random.default_rng(808)
    agree = total = rejected = weak_rejected = 0
    for _ in range(3000):
        D, p, q = hard_swap_case(rng)
        if oracle.validate(D) != 0:
            continue
        k = p + q
        st, Dn, Qn = oracle.swap(D, 0, p, q, Q=np.eye(k))
        sel = np.zeros(k, np.int32)
        sel[p:] = 1
        info = lapack.dtrsen(sel, D, np.eye(k), job="N")[-1]
        total += 1
        agree += int(st == info)
        rejected += st
        if st == 0:
            assert is_standard(Dn)
            assert np.linalg.norm(Qn.T @ D @ Qn - Dn) <= 50 * EPS * np.linalg.norm(D)
        else:
            assert np.array_equal(Dn, D)
        # the weak test alone must already guarantee a small backward error
        stw, Dw, Qw = oracle.swap(D, 0, p, q, Q=np.eye(k), strong=False)
        if stw == 0:
            assert np.linalg.norm(Qw.T @ D @ Qw - Dw) <= 100 * EPS * np.linalg.norm(D)
        else:
            weak_rejected += 1
    assert weak_rejected > 20
    assert total > 2000
    assert rejected > 50
    assert agree >= 0.99 * total


# ------------------------------------------------------- brute force, tiny n

def spectral_basis(S, want):
    """Real basis of the invariant subspace of the eigenvalues `want`
    (list of complex, conjugates included), from numpy eigenvectors."""
    w, V = np.linalg.eig(S)
    cols = []
    used = np.zeros(w.size, dtype=bool)
    for lam in want:
        if lam.imag < 0:
            continue
        d = np.abs(w - lam)
        d[used] = np.inf
        i = int(np.argmin(d))
        used[i] = True
        if lam.imag == 0:
            cols.append(V[:, i].real)
        else:
            cols += [V[:, i].real, V[:, i].imag]
    return np.array(cols).T if cols else np.zeros((S.shape[0], 0))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_bruteforce_all_selections(n):
    rng = np.random.default_rng(600 + n)
    for trial in range(2):
        S, sizes = well_conditioned_schur(n, rng, upper_scale=0.5)
        starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
        for mask in itertools.product([0, 1], repeat=len(sizes)):
            sel = np.zeros(n, dtype=np.int32)
            for b, on in enumerate(mask):
                if on:
                    sel[starts[b]:starts[b] + sizes[b]] = 1
            r = oracle.reorder(S, np.eye(n), sel)
            assert r["status"] == 0
            want, m = expected_order(S, sel)
            assert r["m"] == m
            got = block_eigs(r["S"])
            assert match_eigs(got, want, 0) <= 1e-12
            assert is_standard(r["S"])
            assert orth_err(r["Q"]) <= 50 * n * EPS
            assert residual(S, r["S"], r["Q"]) <= 50 * n * EPS
            if 0 < m < n:
                B = spectral_basis(S, list(want[:m]))
                sep = dtrsen_sep(S, sel)
                cond = np.linalg.norm(S) / sep
                assert sin_angle(r["Q"][:, :m], B) <= 1e-12 * cond


# --------------------------------------------- LAPACK dtrsen cross-check

@pytest.mark.parametrize("n,seed,frac", [(12, 1, 0.5), (50, 2, 0.3), (200, 3, 0.35), (400, 0, 0.3)])
def test_dtrsen_crosscheck(n, seed, frac):
    S, Q, sel = si.reorder_problem(n, seed, select_frac=frac, q="householder")
    r = oracle.reorder(S, Q, sel, abort=True)
    ts, qs, wr2, wi2, m2, s_, sep_, info = lapack.dtrsen(sel, S, Q, job="N")
    assert info == 0 and r["status"] == 0
    assert r["m"] == m2
    got = r["wr"] + 1j * r["wi"]
    want = wr2 + 1j * wi2
    assert match_eigs(got, want, 0) <= 1e-10
    m = r["m"]
    # subspace agreement (both backward stable); cond-free bound is checked
    # on the well-conditioned case below
    assert sin_angle(r["Q"][:, :m], qs[:, :m]) <= 1e-8


@pytest.mark.parametrize("n,seed", [(60, 11), (150, 12)])
def test_dtrsen_crosscheck_well_conditioned(n, seed):
    rng = np.random.default_rng(seed)
    S, sizes = well_conditioned_schur(n, rng)
    S = np.asfortranarray(S)
    sel = si.selection(sizes, 0.4, rng)
    Q = si.householder_q(n, rng, 16)
    r = oracle.reorder(S, Q, sel, abort=True)
    ts, qs, wr2, wi2, m2, s_, sep_, info = lapack.dtrsen(sel, S, Q, job="N")
    assert info == 0 and r["status"] == 0
    m = r["m"]
    cond = np.linalg.norm(S) / dtrsen_sep(S, sel)
    assert match_eigs(r["wr"] + 1j * r["wi"], wr2 + 1j * wi2, 0) <= 1e-12
    assert sin_angle(r["Q"][:, :m], qs[:, :m]) <= 1e-10 * cond
    assert cond < 1e8   # the bound above is meaningful here


# ----------------------------------------------------------- invariants

@pytest.mark.parametrize("name", ["n400"])
def test_invariants_n400(name):
    S, Q, sel = si.config(name)
    n = S.shape[0]
    A = Q @ S @ Q.T
    r = oracle.reorder(S, Q, sel)
    assert r["status"] == 0
    want, m = expected_order(S, sel)
    got = block_eigs(r["S"])
    assert match_eigs(got, want, 0) <= 1e-10
    assert np.allclose(np.sort_complex(got), np.sort_complex(block_eigs(S)), rtol=1e-10)
    assert r["sel"][:m].all() and not r["sel"][m:].any()
    assert is_standard(r["S"])
    assert orth_err(r["Q"]) <= 50 * n * EPS
    assert residual(A, r["S"], r["Q"]) <= 50 * n * EPS


def test_rejection_semantics():
    """Clustered spectra with non-normal 2x2 blocks (kappa = 1e6) force
    rejections: CONTINUE keeps a valid similarity and counts them; ABORT
    stops at the first, as LAPACK's dtrsen does (info = 1)."""
    n = 300
    S, Q, sel = si.reorder_problem(n, 3, select_frac=0.5, clusters=True, spread=1e-6,
                                   kappa=1e6)
    A = Q @ S @ Q.T
    r = oracle.reorder(S, Q, sel)
    assert r["status"] > 0 and r["nrej"] == r["status"]
    assert is_standard(r["S"])
    assert residual(A, r["S"], r["Q"]) <= 50 * n * EPS
    assert orth_err(r["Q"]) <= 50 * n * EPS
    # the eigenvalue multiset is preserved even when the order is partial.
    # With |b|/|c| ~ 1e12 inside the 2x2 blocks, a perturbation of 1e-16 |b|
    # in c moves sqrt(-bc) by ~1e-4 relative: that is the attainable accuracy
    # of these eigenvalues, so the check allows 1e-3.
    a, b = block_eigs(S), block_eigs(r["S"])
    cost = np.abs(a[:, None] - b[None, :])
    i, j = linear_sum_assignment(cost)
    assert cost[i, j].max() <= 1e-3
    ra = oracle.reorder(S, Q, sel, abort=True)
    assert ra["status"] == 1
    ts, qs, wr2, wi2, m2, s_, sep_, info = lapack.dtrsen(sel, S, Q, job="N")
    assert info == 1
    # same partial result as LAPACK up to the rejection
    assert match_eigs(ra["wr"] + 1j * ra["wi"], wr2 + 1j * wi2, 0) <= 1e-8


def test_edge_cases():
    # n = 0 and n = 1
    assert oracle.reorder(np.zeros((0, 0)), None, np.zeros(0, np.int32))["status"] == 0
    r = oracle.reorder(np.array([[2.0]]), np.eye(1), np.array([1], np.int32))
    assert r["status"] == 0 and r["m"] == 1 and r["S"][0, 0] == 2.0
    # nothing selected / everything selected: S unchanged
    S, Q, sel = si.reorder_problem(30, 5)
    for s in (np.zeros(30, np.int32), np.ones(30, np.int32)):
        r = oracle.reorder(S, Q, s)
        assert r["status"] == 0 and np.array_equal(r["S"], S) and np.array_equal(r["Q"], Q)
    # half of a 2x2 block selects the whole pair
    S2 = np.array([[1.0, 3.0, 0.5], [0.0, 0.2, 1.0], [0.0, -2.0, 0.2]], order="F")
    r = oracle.reorder(S2, np.eye(3), np.array([0, 0, 1], np.int32))
    assert r["m"] == 2 and r["S"][1, 0] != 0.0 and abs(r["S"][2, 2] - 1.0) < 1e-14
    # Q may be omitted
    r = oracle.reorder(S, None, sel)
    assert r["status"] == 0 and r["Q"] is None
    # invalid inputs
    bad = S.copy(order="F")
    bad[5, 2] = 1.0
    assert oracle.reorder(bad, None, sel)["status"] == -2
    nonstd = np.array([[1.0, 1.0], [-1.0, 2.0]], order="F")  # unequal diagonal
    assert oracle.reorder(nonstd, None, np.array([1, 0], np.int32))["status"] == -2
