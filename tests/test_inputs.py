"""The seeded input generator: the laws the workloads state (these inputs
feed both the oracle and the GPU path, so their shape is checked here)."""
import numpy as np

import schur_inputs as si
from tests.helpers import blocks, expected_order, is_standard


def test_schur_form_laws():
    rng = np.random.default_rng(3)
    S, sizes = si.schur_form(500, rng)
    assert is_standard(S)
    assert int(np.sum(sizes)) == 500
    n1 = int(np.sum(sizes == 1))
    assert n1 == round(0.6 * 500) or n1 == round(0.6 * 500) + 1
    for j, sz in blocks(S):
        if sz == 2:
            b, c = S[j, j + 1], S[j + 1, j]
            assert 0.1 <= abs(b) <= 2 and 0.1 <= abs(c) <= 2 and b * c < 0


def test_selection_counts_and_pairs():
    rng = np.random.default_rng(4)
    S, sizes = si.schur_form(301, rng)
    sel = si.selection(sizes, 0.35, rng)
    assert round(0.35 * 301) <= sel.sum() <= round(0.35 * 301) + 1
    for j, sz in blocks(S):
        if sz == 2:
            assert sel[j] == sel[j + 1]


def test_householder_q_orthogonal():
    Q = si.householder_q(200, np.random.default_rng(5), 64)
    assert np.linalg.norm(Q.T @ Q - np.eye(200)) < 1e-12


def test_batch_and_request_laws():
    b = si.batch_problems(500, 0, 32, 512)
    ns = np.array([x[0] for x in b])
    ps = np.array([x[1] for x in b])
    assert ns.min() >= 32 and ns.max() <= 512 and 0.2 <= ps.min() and ps.max() <= 0.6
    r = si.request_stream(2000, 0, 64, 8192, rate=10.0)
    t = np.array([x[0] for x in r])
    n = np.array([x[1] for x in r])
    assert np.all(np.diff(t) > 0)
    assert 64 <= n.min() and n.max() <= 8192
    # log-uniform: the median order is near sqrt(64 * 8192) = 724
    assert 500 < np.median(n) < 1050
    # Poisson at 10 per second: mean gap 0.1 s
    assert abs(np.mean(np.diff(t)) - 0.1) < 0.01


def test_serve_requests_are_standard_subblocks():
    base = si.serve_base(1024, 1)
    for _, n, p, sd in si.request_stream(40, 2, 16, 1024):
        S, Q, sel = si.serve_request(base, n, p, sd)
        m = S.shape[0]
        assert min(n, 1024) <= m <= min(n, 1024) + 1
        assert is_standard(S)
        assert np.linalg.norm(Q.T @ Q - np.eye(m)) < 1e-12
        want, k = expected_order(S, sel)
        assert abs(k - round(p * m)) <= 1
        # the sub-block is the base form's principal block at some offset
        k0 = next(i for i in range(1025 - m) if np.array_equal(base[0][i:i + m, i:i + m], S))
        assert k0 == 0 or base[0][k0, k0 - 1] == 0.0


def test_generalized_pair_laws():
    """(S, T): T upper triangular with diagonal in [0.5, 2]; a 1x1 block of
    S is lambda t_jj; a 2x2 block is T_b M with M standardized, so the
    pencil block has M's complex pair; Q and Z orthogonal."""
    from tests.helpers import gen_block_eigs, is_gen_schur
    S, T, Q, Z, sel = si.gen_problem(300, 5, select_frac=0.35, reflectors=8)
    assert is_gen_schur(S, T)
    d = np.diag(T)
    assert np.all((d >= 0.5) & (d <= 2.0))
    ev = gen_block_eigs(S, T)
    for j, sz in blocks(S):
        if sz == 2:
            M = np.linalg.solve(T[j:j + 2, j:j + 2], S[j:j + 2, j:j + 2])
            assert abs(M[0, 0] - M[1, 1]) <= 1e-12 * max(1.0, abs(M[0, 0]))
            assert M[0, 1] * M[1, 0] < 0
            assert abs(ev[j].imag) > 0 and np.isclose(ev[j], np.conj(ev[j + 1]))
            assert sel[j] == sel[j + 1]
    for X in (Q, Z):
        assert np.linalg.norm(X.T @ X - np.eye(300)) <= 1e-12
    assert round(0.35 * 300) <= sel.sum() <= round(0.35 * 300) + 1


def test_hessenberg_sweep_inputs():
    """H upper Hessenberg with N(0,1) entries; shifts in pairs, alternately
    a conjugate pair with imaginary part in [0.1, 1] and two real shifts."""
    H, Q, sh = si.hessenberg_problem(200, 2, nshifts=8, reflectors=8)
    assert np.all(np.tril(H, -2) == 0.0) and np.all(np.diag(H, -1) != 0.0)
    assert len(sh) == 8
    for b in range(4):
        a1, a2 = sh[2 * b], sh[2 * b + 1]
        if b % 2 == 0:
            assert a1 == np.conj(a2) and 0.1 <= a1.imag <= 1.0
        else:
            assert a1.imag == 0.0 and a2.imag == 0.0
    assert np.linalg.norm(Q.T @ Q - np.eye(200)) <= 1e-12
