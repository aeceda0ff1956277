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
