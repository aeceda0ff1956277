"""Host-side check of the generalized path's structure (runs without a
GPU): the planner's windows, and inside each window the wavefront of swaps
(every selected block whose upper neighbour is unselected swaps in the same
step; all left products, then all right products; UQ and UZ accumulated),
then UQ / UZ applied to the rows to the right, the columns above, Q and Z --
replayed in numpy with the oracle's local swap -- give the oracle's
reordering: the same eigenvalue order and deflating subspaces, a valid
equivalence."""
import numpy as np
import pytest

import oracle
import schur_inputs as si
import paper_1905_04975_gb300 as g
from paper_1905_04975_gb300 import build as gbuild
from tests.helpers import (EPS, gen_block_eigs, gen_expected_order, is_gen_schur, match_eigs,
                           orth_err, pair_residual, sin_angle)


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    return g.load()


def block_starts(S, lo, hi):
    """bst[i] for rows lo..hi-1: a block starts at i."""
    return [i == lo or S[i, i - 1] == 0.0 for i in range(lo, hi)]


def replay(S, T, Q, Z, select, window, chain):
    S, T, Q, Z = (X.copy() for X in (S, T, Q, Z))
    n = S.shape[0]
    sub = np.array([1 if (i + 1 < n and S[i + 1, i] != 0.0) else 0 for i in range(n)], np.uint8)
    sel = np.asarray(select, bool).copy()
    for i in range(n - 1):
        if sub[i]:
            sel[i] = sel[i + 1] = sel[i] or sel[i + 1]
    wins, _, _ = g.plan(sub, sel.astype(np.int32), window=window, chain=chain)
    for s, e in wins:
        w = e - s
        A, B = S[s:e, s:e], T[s:e, s:e]   # views: updated in place
        UQ, UZ = np.eye(w), np.eye(w)
        ls = sel[s:e]                      # view
        while True:
            bst = block_starts(S, s, e)
            swaps = []
            for t in range(1, w):
                if not bst[t] or not ls[t]:
                    continue
                ja = t - 1 if bst[t - 1] else t - 2
                if ls[ja]:
                    continue
                p = t - ja
                q = 2 if (t + 1 < w and not bst[t + 1]) else 1
                swaps.append((ja, p, q))
            if not swaps:
                break
            done = []
            for ja, p, q in swaps:
                k = p + q
                st, Qs, Zs, NA, NB = oracle.gen_swap_local(A[ja:ja + k, ja:ja + k],
                                                           B[ja:ja + k, ja:ja + k], p, q)
                assert st == 0
                A[ja:ja + k, ja:ja + k] = NA
                B[ja:ja + k, ja:ja + k] = NB
                done.append((ja, k, q, Qs, Zs))
            for ja, k, q, Qs, Zs in done:        # left: rows of the block, columns to the right
                A[ja:ja + k, ja + k:] = Qs.T @ A[ja:ja + k, ja + k:]
                B[ja:ja + k, ja + k:] = Qs.T @ B[ja:ja + k, ja + k:]
            for ja, k, q, Qs, Zs in done:        # right: columns of the block, rows above
                A[:ja, ja:ja + k] = A[:ja, ja:ja + k] @ Zs
                B[:ja, ja:ja + k] = B[:ja, ja:ja + k] @ Zs
                UQ[:, ja:ja + k] = UQ[:, ja:ja + k] @ Qs
                UZ[:, ja:ja + k] = UZ[:, ja:ja + k] @ Zs
                ls[ja:ja + q] = True
                ls[ja + q:ja + k] = False
        for X in (S, T):
            X[s:e, e:] = UQ.T @ X[s:e, e:]
            X[:s, s:e] = X[:s, s:e] @ UZ
        Q[:, s:e] = Q[:, s:e] @ UQ
        Z[:, s:e] = Z[:, s:e] @ UZ
    return S, T, Q, Z


@pytest.mark.parametrize("n,seed,window,chain", [(12, 1, 8, 3), (60, 2, 16, 6), (150, 3, 32, 12),
                                                  (200, 4, 64, 32)])
def test_windowed_wavefront_matches_oracle(n, seed, window, chain):
    S, T, Q, Z, sel = si.gen_problem(n, seed, select_frac=0.45, reflectors=8)
    Sr, Tr, Qr, Zr = replay(S, T, Q, Z, sel, window, chain)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    assert ref["status"] == 0
    want, m = gen_expected_order(S, T, sel)
    assert is_gen_schur(Sr, Tr)
    got = gen_block_eigs(Sr, Tr)
    assert match_eigs(got, want, 0) <= 1e-10
    assert match_eigs(got, ref["eigs"], 0) <= 1e-10
    assert orth_err(Qr) <= 20 * n * EPS and orth_err(Zr) <= 20 * n * EPS
    assert pair_residual(Q @ S @ Z.T, Q @ T @ Z.T, Sr, Tr, Qr, Zr) <= 20 * n * EPS
    if 0 < m < n:
        assert sin_angle(Qr[:, :m], ref["Q"][:, :m]) <= 1e-8
        assert sin_angle(Zr[:, :m], ref["Z"][:, :m]) <= 1e-8
