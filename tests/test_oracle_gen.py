"""Pins of the generalized reordering oracle (Eq. 7, second form: (S, T) =
Q3 (S_hat, T_hat) Z3^T): an independent library (LAPACK's reordering of a
generalized Schur form through scipy.linalg.ordqz, and its generalized
eigenvalues), the reduction to the standard problem (T = I), a closed form
for two 1x1 blocks, and invariants (orthogonality, backward error, exact
structure, eigenvalue order)."""
import numpy as np
import pytest

import oracle
import schur_inputs as si
from tests.helpers import (EPS, blocks, gen_block_eigs, gen_expected_order, is_gen_schur,
                           match_eigs, orth_err, pair_residual, sin_angle)

scipy_linalg = pytest.importorskip("scipy.linalg")


def run(S, T, Q, Z, sel, **kw):
    A, B = Q @ S @ Z.T, Q @ T @ Z.T
    r = oracle.gen_reorder(S, T, Q, Z, sel, **kw)
    return A, B, r


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (7, 3), (12, 4), (60, 5), (200, 6)])
def test_invariants_and_order(n, seed):
    S, T, Q, Z, sel = si.gen_problem(n, seed, select_frac=0.5, reflectors=8)
    assert oracle.gen_validate(S, T) == 0
    A, B, r = run(S, T, Q, Z, sel)
    assert r["status"] == 0
    want, m = gen_expected_order(S, T, sel)
    assert r["m"] == m
    assert is_gen_schur(r["S"], r["T"])
    assert oracle.gen_validate(r["S"], r["T"]) == 0
    # eigenvalues read by the oracle agree with LAPACK on the output blocks
    got = gen_block_eigs(r["S"], r["T"])
    assert match_eigs(r["eigs"], got, 0) <= 1e-12
    assert match_eigs(got, want, 0) <= 1e-10
    assert orth_err(r["Q"]) <= 20 * max(n, 1) * EPS
    assert orth_err(r["Z"]) <= 20 * max(n, 1) * EPS
    assert pair_residual(A, B, r["S"], r["T"], r["Q"], r["Z"]) <= 20 * max(n, 1) * EPS


def test_against_lapack_ordqz():
    """The leading left and right deflating subspaces for the selected
    eigenvalues equal those of LAPACK's reordering (scipy ordqz) of the same
    pencil.  The coupling above the diagonal blocks of S is scaled down so
    that the subspaces are well conditioned."""
    n = 40
    S, T, Q, Z, sel = si.gen_problem(n, 11, select_frac=0.5, reflectors=8)
    mask = np.triu(np.ones((n, n), dtype=bool), 1)
    for j, sz in blocks(S):
        if sz == 2:
            mask[j, j + 1] = False
    S[mask] *= 0.05
    T[mask] *= 0.05
    A, B, r = run(S, T, Q, Z, sel)
    assert r["status"] == 0
    m = r["m"]
    want = r["eigs"][:m]

    def chosen(alpha, beta):
        lam = alpha / beta
        return np.array([np.min(np.abs(want - l)) <= 1e-8 * max(1.0, abs(l)) for l in lam])

    AA, BB, alpha, beta, QL, ZL = scipy_linalg.ordqz(A, B, sort=chosen, output="real")
    lam = alpha / beta
    assert np.sort_complex(lam[:m]).round(8).tolist() == np.sort_complex(want).round(8).tolist()
    assert sin_angle(r["Z"][:, :m], ZL[:, :m]) <= 1e-10
    assert sin_angle(r["Q"][:, :m], QL[:, :m]) <= 1e-10


def test_generalized_eigenvalues_against_lapack():
    """Eigenvalues read from the blocks of the input equal LAPACK's
    generalized eigenvalues of the full pencil (as sets); the coupling above
    the blocks is scaled down so that every eigenvalue is well conditioned."""
    n = 50
    S, T, Q, Z, _ = si.gen_problem(n, 3, reflectors=8)
    mask = np.triu(np.ones((n, n), dtype=bool), 1)
    for j, sz in blocks(S):
        if sz == 2:
            mask[j, j + 1] = False
    S[mask] *= 0.05
    T[mask] *= 0.05
    ours = oracle.gen_eigenvalues(S, T)
    ref = scipy_linalg.eigvals(Q @ S @ Z.T, Q @ T @ Z.T)
    for l in ours:
        assert np.min(np.abs(ref - l)) <= 1e-9 * max(1.0, abs(l))


def test_reduces_to_standard_reordering():
    """With T = I and Z = Q the pair problem is the standard one: same
    eigenvalue order and leading invariant subspace as the standard oracle,
    Z = Q and T = I to rounding."""
    n = 50
    S, Q, sel = si.reorder_problem(n, 21, select_frac=0.4, q="householder", reflectors=8)
    T = np.eye(n)
    A, B, r = run(S, T, Q, Q.copy(), sel)
    ref = oracle.reorder(S, Q, sel)
    assert r["status"] == 0 and ref["status"] == 0
    assert match_eigs(r["eigs"], ref["wr"] + 1j * ref["wi"], 0) <= 1e-10
    m = r["m"]
    assert sin_angle(r["Q"][:, :m], ref["Q"][:, :m]) <= 1e-10
    assert np.linalg.norm(r["Q"] - r["Z"]) <= 100 * n * EPS
    assert np.linalg.norm(r["T"] - np.eye(n)) <= 100 * n * EPS


def test_two_1x1_blocks_closed_form():
    """Pencil [[a11, a12], [0, a22]], [[b11, b12], [0, b22]]: after the
    swap the first column of Z is the right eigenvector of lambda2 =
    a22/b22, x = (-(b22 a12 - a22 b12) / (b22 a11 - a22 b11), 1), and the
    diagonal ratios are exchanged."""
    a11, a12, a22, b11, b12, b22 = 0.7, -1.3, -0.4, 1.5, 0.25, 0.8
    S = np.array([[a11, a12], [0.0, a22]])
    T = np.array([[b11, b12], [0.0, b22]])
    r = oracle.gen_reorder(S, T, np.eye(2), np.eye(2), [0, 1])
    assert r["status"] == 0 and r["nswaps"] == 1
    x = np.array([-(b22 * a12 - a22 * b12) / (b22 * a11 - a22 * b11), 1.0])
    x /= np.linalg.norm(x)
    z = r["Z"][:, 0]
    assert abs(abs(z @ x) - 1.0) <= 4 * EPS
    S2, T2 = r["S"], r["T"]
    assert S2[1, 0] == 0.0 and T2[1, 0] == 0.0
    assert abs(S2[0, 0] / T2[0, 0] - a22 / b22) <= 8 * EPS
    assert abs(S2[1, 1] / T2[1, 1] - a11 / b11) <= 8 * EPS
    # the left vector: Q's first column spans A x (and B x)
    q = r["Q"][:, 0]
    ax = np.array([[a11, a12], [0, a22]]) @ x
    assert abs(abs(q @ ax) / np.linalg.norm(ax) - 1.0) <= 8 * EPS


@pytest.mark.parametrize("p,q", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_local_swap_every_type(p, q):
    """One swap on a k x k pair: Qs, Zs orthogonal, Qs^T (A, B) Zs block
    upper triangular with the q x q block's eigenvalues first, T part upper
    triangular, backward error at rounding level."""
    rng = np.random.default_rng(100 + 10 * p + q)
    frac = {2: 1.0, 3: 0.34, 4: 0.0}[p + q]
    for _ in range(200):
        S, T, sizes = si.gen_schur_pair(p + q, rng, frac_1x1=frac)
        if list(sizes) == [p, q]:
            break
    assert list(sizes) == [p, q]
    st, Qs, Zs, NA, NB = oracle.gen_swap_local(S, T, p, q)
    assert st == 0
    k = p + q
    assert orth_err(Qs) <= 8 * EPS and orth_err(Zs) <= 8 * EPS
    assert np.all(NA[q:, :q] == 0.0) and np.all(np.tril(NB, -1) == 0.0)
    assert np.linalg.norm(Qs @ NA @ Zs.T - S) <= 50 * EPS * np.linalg.norm(S)
    assert np.linalg.norm(Qs @ NB @ Zs.T - T) <= 50 * EPS * np.linalg.norm(T)
    before = gen_block_eigs(S, T)
    after = gen_block_eigs(NA, NB)
    assert match_eigs(after, np.concatenate([before[p:], before[:p]]), 0) <= 1e-12


@pytest.mark.parametrize("p,q", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_generalized_sylvester_residual(p, q):
    rng = np.random.default_rng(7 * p + q)
    k = p + q
    A = np.triu(rng.standard_normal((k, k)))
    B = np.triu(rng.standard_normal((k, k))) + 2 * np.eye(k)
    R, L, g = oracle.gen_sylvester(A, B, p, q)
    assert g == 1.0
    ra = A[:p, :p] @ R - L @ A[p:, p:] + g * A[:p, p:]
    rb = B[:p, :p] @ R - L @ B[p:, p:] + g * B[:p, p:]
    scale = max(1.0, np.abs(R).max(), np.abs(L).max())
    assert np.abs(ra).max() <= 50 * EPS * scale * np.abs(A).max()
    assert np.abs(rb).max() <= 50 * EPS * scale * np.abs(B).max()


def test_equal_eigenvalues_and_selection_rules():
    """Two 1x1 blocks with equal generalized eigenvalues are already in
    order (nothing changes); a 2x2 block is moved whole when one of its
    positions is selected; nothing selected changes nothing."""
    S = np.array([[2.0, 1.0], [0.0, 1.0]])
    T = np.array([[1.0, 3.0], [0.0, 0.5]])
    r = oracle.gen_reorder(S, T, np.eye(2), np.eye(2), [0, 1])
    assert r["status"] == 0 and np.array_equal(r["S"], S) and np.array_equal(r["T"], T)
    S, T, Q, Z, _ = si.gen_problem(30, 9, reflectors=4)
    r0 = oracle.gen_reorder(S, T, Q, Z, np.zeros(30, np.int32))
    assert np.array_equal(r0["S"], S) and np.array_equal(r0["Q"], Q)
    two = [j for j, sz in blocks(S) if sz == 2]
    j = two[-1]
    sel = np.zeros(30, np.int32)
    sel[j + 1] = 1
    r1 = oracle.gen_reorder(S, T, Q, Z, sel)
    assert r1["m"] == 2
    ev = gen_block_eigs(S, T)
    assert match_eigs(r1["eigs"][:2], ev[j:j + 2], 0) <= 1e-10


def ill_conditioned_pair():
    """Two 2x2 blocks with eigenvalues 1.4e-8 apart and strongly non-normal
    standardized parts (|b| / |c| ~ 1e15): a swap that cannot be done
    stably.  T's 2x2 blocks are diagonal so LAPACK takes the pair as is."""
    rng = np.random.default_rng(1)
    d, kap, cpl = 10 ** rng.uniform(-14, -2), 10 ** rng.uniform(0, 8), 10 ** rng.uniform(-3, 3)
    a, b, c = rng.standard_normal(), rng.uniform(0.1, 2), -rng.uniform(0.1, 2)
    M1 = np.array([[a, b * kap], [c / kap, a]])
    M2 = np.array([[a + d, b * kap], [c / kap, a + d]])
    T = np.diag(rng.uniform(0.5, 2, 4))
    T[0, 2:] = rng.standard_normal(2)
    T[1, 2:] = rng.standard_normal(2)
    S = np.zeros((4, 4))
    S[:2, :2] = T[:2, :2] @ M1
    S[2:, 2:] = T[2:, 2:] @ M2
    S[:2, 2:] = rng.standard_normal((2, 2)) * cpl
    return np.asfortranarray(S), np.asfortranarray(T)


def test_rejected_swap_changes_nothing():
    """The ill-conditioned swap is rejected by the weak test alone (LAPACK's
    dtgexc refuses it too); the reordering then reports one rejection and
    leaves S, T, Q, Z exactly as they were."""
    S, T = ill_conditioned_pair()
    st_weak, *_ = oracle.gen_swap_local(S, T, 2, 2, strong=False)
    assert st_weak == 1
    info = scipy_linalg.lapack.dtgexc(S, T, np.eye(4), np.eye(4), 3, 1)[-1]
    assert info != 0
    Q = np.eye(4)
    r = oracle.gen_reorder(S, T, Q, Q, [0, 0, 1, 1])
    assert r["status"] == 1 and r["nrej"] == 1 and r["nswaps"] == 0
    assert np.array_equal(r["S"], S) and np.array_equal(r["T"], T)
    assert np.array_equal(r["Q"], Q) and np.array_equal(r["Z"], Q)


def test_eigenvalues_of_a_real_pair_block():
    """A 2x2 block whose pencil has two real eigenvalues (which rounding in a
    swap could produce) gives both roots, the larger first, as LAPACK's
    generalized eigenvalues of that block; a 1x1 block with t = 0 gives an
    infinite eigenvalue."""
    Tb = np.array([[1.5, 0.3], [0.0, 0.8]])
    M = np.array([[1.0, 2.0], [0.5, -0.7]])          # real eigenvalues
    S = np.zeros((3, 3))
    T = np.zeros((3, 3))
    S[:2, :2] = Tb @ M
    T[:2, :2] = Tb
    S[2, 2], T[2, 2] = 1.0, 0.0
    S[0, 2], T[0, 2] = 0.4, 0.2
    ev = oracle.gen_eigenvalues(S, T)
    ref = np.sort(np.linalg.eigvals(M).real)[::-1]
    assert np.allclose(ev[:2].real, ref, rtol=1e-14, atol=0) and np.all(ev[:2].imag == 0)
    assert np.isinf(ev[2].real)
