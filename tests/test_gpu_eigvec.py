"""GPU eigenvectors of a real Schur form (Eq. 5) with back-transformation
(Eq. 6) and overflow protection, through gbr_eigenvectors, against the CPU
oracle (same definition, same normalization): element-wise on the
normalized vectors, plus residuals ||A x - lambda x|| of the GPU result."""
import numpy as np
import pytest

import oracle
import schur_inputs as si

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


def run(gbr, S, Q, select):
    Sd = gbr.to_device(S)
    Qd = gbr.to_device(Q) if Q is not None else None
    X, ns = gbr.eigenvectors(Sd, Qd, select, with_scalings=True)
    torch.cuda.synchronize()
    return gbr.to_host(X), ns


def residuals(A, X, kinds, lams):
    out, c = [], 0
    while c < X.shape[1]:
        if kinds[c] == 0:
            x = X[:, c].astype(complex)
            c += 1
        else:
            x = X[:, c] + 1j * X[:, c + 1]
            c += 2
        out.append(np.linalg.norm(A @ x - lams[c - 1] * x) / (np.linalg.norm(A) * np.linalg.norm(x)))
    return np.array(out)


CASES = [("n1", 1, None), ("n2", 2, None), ("n7", 7, None), ("n60", 60, "sub"),
         ("ragged515", 515, None), ("n400", 400, "sub")]


@pytest.mark.parametrize("name,n,sel", CASES)
@pytest.mark.parametrize("withq", [False, True])
def test_eigvec_matches_oracle(gbr, name, n, sel, withq):
    if name == "n400":
        S, Q, _ = si.config("n400")
        Q = si.householder_q(n, np.random.default_rng(3), 16)
    else:
        S, Q, _ = si.reorder_problem(n, n + 1, select_frac=0.4, q="householder", reflectors=8)
    select = None
    if sel == "sub":
        select = np.zeros(n, dtype=np.int32)
        select[::3] = 1
    Qu = Q if withq else None
    Xg, ns = run(gbr, S, Qu, select)
    Xo, kinds, lams, nso = oracle.eigenvectors(S, Qu, select)
    assert Xg.shape == Xo.shape
    # same definition and normalization: agreement to the rounding of the
    # back substitution (FMA on the GPU, none in the oracle), amplified by
    # the conditioning of each vector
    assert np.max(np.abs(Xg - Xo)) <= 1e-9
    A = Q @ S @ Q.T if withq else S
    assert np.all(residuals(A, Xg, kinds, lams) <= 50 * n * EPS)
    assert np.array_equal(ns, nso)


def growth_matrix(kind, n):
    T = np.zeros((n, n))
    for i in range(n):
        if kind == "gaps":
            T[i, i] = 1.0 + i * 2.0 ** -30
            T[i, i + 1:] = 2.0 ** 30 * (1 + (np.arange(i + 1, n) % 3))
        elif kind == "tiny pivots":
            T[i, i] = i * 2.0 ** -600
            T[i, i + 1:] = 1.0 + (np.arange(i + 1, n) % 2)
        else:
            T[i, i] = 1.0 + i
            T[i, i + 1:] = 2.0 ** 300 * (1 + (np.arange(i + 1, n) % 3))
    return T


@pytest.mark.parametrize("kind,n", [("gaps", 40), ("tiny pivots", 12), ("couplings", 12)])
def test_overflow_protection(gbr, kind, n):
    """Growth patterns that overflow without scaling: the GPU scales (exact
    powers of two) and matches the oracle, which matches exact rationals."""
    T = growth_matrix(kind, n)
    Xg, ns = run(gbr, T, None, None)
    Xo, _, _, nso = oracle.eigenvectors(T)
    assert np.all(np.isfinite(Xg))
    assert ns[n - 1] > 0
    assert np.allclose(Xg, Xo, rtol=1e-12, atol=1e-300)


def test_n4000_workload_all_vectors(gbr):
    """All 4000 eigenvectors of the n = 4000 Schur form, back-transformed by
    its Q (64 reflectors): residual of every vector, oracle on a sample of
    columns."""
    S, Q, _ = si.config("n4000")
    n = S.shape[0]
    Xg, ns = run(gbr, S, Q, None)
    kinds, lams = oracle.eig_columns(S)
    assert Xg.shape == (n, n) and np.all(np.isfinite(Xg))
    A = Q @ S @ Q.T
    cols = np.arange(0, n, 97)
    # residuals on a sample of vectors (whole pairs)
    sample = []
    for c in cols:
        c0 = c - 1 if kinds[c] == 2 else c
        sample += [c0] if kinds[c0] == 0 else [c0, c0 + 1]
    sample = sorted(set(sample))
    Xs = Xg[:, sample]
    ks = kinds[sample]
    ls = lams[sample]
    assert np.all(residuals(A, Xs, ks, ls) <= 50 * n * EPS)
    # oracle on the positions of the sampled columns
    select = np.zeros(n, dtype=np.int32)
    pos, c, j = [], 0, 0
    while j < n:
        nb = 2 if (j + 1 < n and S[j + 1, j] != 0) else 1
        if any(c + t in sample for t in range(nb)):
            select[j] = 1
        c += nb
        j += nb
    Xo, _, _, _ = oracle.eigenvectors(S, Q, select)
    assert Xo.shape[1] == len(sample)
    assert np.max(np.abs(Xs - Xo)) <= 1e-9
