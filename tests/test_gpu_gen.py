"""GPU reordering of a generalized Schur form (S, T) with Q and Z (Eq. 7,
second form) through gbr_reorder_gen, against the CPU oracle.

As for the standard form, the reordered pair is unique only up to the signs
of the Schur vectors and the basis inside each 2x2 block, so parity compares
what is unique:
  * the generalized eigenvalue order on the diagonal (1e-10 relative),
  * the leading left and right deflating subspaces (span Q[:, :m] and
    span Z[:, :m]) against the oracle's: sine of the largest principal angle
    <= 1e-10 cond, cond = ||(S, T)||_F / Dif (LAPACK's estimate),
and checks that the rest is valid: exact zeros below the quasi-diagonal of
S and below the diagonal of T, ||Q^T Q - I||, ||Z^T Z - I|| and the
backward errors ||A - Q S Z^T|| / ||A||, ||B - Q T Z^T|| / ||B|| within
50 n eps.
"""
import numpy as np
import pytest
from scipy.linalg import lapack

import oracle
import schur_inputs as si
from tests.helpers import (EPS, gen_block_eigs, gen_expected_order, is_gen_schur, match_eigs,
                           orth_err, pair_residual, sin_angle)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def run_gpu(g, S, T, Q, Z, sel, **kw):
    d = [g.to_device(X) if X is not None else None for X in (S, T, Q, Z)]
    r = g.reorder_gen(*d, sel, **kw)
    torch.cuda.synchronize()
    return (r,) + tuple(g.to_host(X) if X is not None else None for X in d)


def dif_cond(S, T, sel, m):
    n = S.shape[0]
    if not (0 < m < n) or n > 600:
        return None
    lw = max(4 * n + 16, 2 * m * (n - m) + 1)
    out = lapack.dtgsen(np.asarray(sel, np.int32), S, T, np.eye(n), np.eye(n), ijob=2,
                        lwork=lw, liwork=max(n + 6, 2 * m * (n - m) + 1))
    dif, info = out[-2], out[-1]
    if info != 0 or np.min(dif) <= 0:
        return None
    return np.sqrt(np.linalg.norm(S) ** 2 + np.linalg.norm(T) ** 2) / np.min(dif)


def check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg, ref=None, order_tol=1e-10):
    n = S.shape[0]
    want, m = gen_expected_order(S, T, sel)
    assert r.m == m
    assert is_gen_schur(Sg, Tg)
    got = gen_block_eigs(Sg, Tg)
    assert match_eigs(r.eigs, got, 0) <= 1e-12
    if r.status == 0:
        assert match_eigs(got, want, 0) <= order_tol
    Qi = Q if Q is not None else np.eye(n)
    Zi = Z if Z is not None else np.eye(n)
    Qo = Qg if Qg is not None else None
    if Qg is not None and Zg is not None:
        assert orth_err(Qg) <= 50 * n * EPS and orth_err(Zg) <= 50 * n * EPS
        assert pair_residual(Qi @ S @ Zi.T, Qi @ T @ Zi.T, Sg, Tg, Qg, Zg) <= 50 * n * EPS
    if ref is not None and r.status == 0 and ref["status"] == 0:
        assert match_eigs(got, ref["eigs"], 0) <= order_tol
        if Qo is not None and 0 < m < n:
            cond = dif_cond(S, T, [1 if x else 0 for x in _pos_sel(S, sel)], m)
            bound = max(1e-10 * cond, 1e-12) if cond else 1e-8
            assert sin_angle(Qg[:, :m], ref["Q"][:, :m]) <= bound
            assert sin_angle(Zg[:, :m], ref["Z"][:, :m]) <= bound


def _pos_sel(S, sel):
    """Per-position selection with 2x2 blocks selected whole."""
    n = S.shape[0]
    s = np.asarray(sel).astype(bool).copy()
    j = 0
    while j < n:
        if j + 1 < n and S[j + 1, j] != 0.0:
            s[j] = s[j + 1] = s[j] or s[j + 1]
            j += 2
        else:
            j += 1
    return s


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 11, 12])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_all_windows(gbr, n, seed):
    S, T, Q, Z, sel = si.gen_problem(n, 10 * n + seed, select_frac=0.5, reflectors=4)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel, window=8, chain=3)
    assert r.status == 0
    check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg, ref)


@pytest.mark.parametrize("name,n,w,m", [("n60", 60, 16, 6), ("n200", 200, 64, 32),
                                        ("n200-narrow", 200, 24, 10), ("g400", 400, 64, 32),
                                        ("ragged515", 515, 64, 30)])
@pytest.mark.parametrize("sched", ["persistent", "sequential"])
def test_matches_oracle(gbr, name, n, w, m, sched):
    if name == "g400":
        S, T, Q, Z, sel = si.gen_config("g400")
    else:
        S, T, Q, Z, sel = si.gen_problem(n, n + 3, select_frac=0.4, reflectors=16)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel, window=w, chain=m, sched=sched)
    assert r.status == 0 and r.stats.swaps == ref["nswaps"]
    check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg, ref)


def test_default_window_is_capped(gbr):
    """Default options ask for w = 128; the pair path runs w = 64, m = 32."""
    S, T, Q, Z, sel = si.gen_problem(300, 5, select_frac=0.5, reflectors=8)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel)
    assert r.status == 0
    check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg, ref)


def test_without_q_and_z(gbr):
    """Q and Z are optional: S and T come out as with them."""
    S, T, Q, Z, sel = si.gen_problem(150, 4, select_frac=0.5, reflectors=8)
    r1, S1, T1, _, _ = run_gpu(gbr, S, T, Q, Z, sel, window=32, chain=12)
    r2, S2, T2, _, _ = run_gpu(gbr, S, T, None, None, sel, window=32, chain=12)
    assert np.array_equal(S1, S2) and np.array_equal(T1, T2)
    assert r1.status == r2.status == 0


def test_host_entry_matches_device_entry(gbr):
    S, T, Q, Z, sel = si.gen_problem(180, 6, select_frac=0.3, reflectors=8)
    r1, S1, T1, Q1, Z1 = run_gpu(gbr, S, T, Q, Z, sel, window=48, chain=20)
    Sh, Th, Qh, Zh = (np.asfortranarray(X.copy()) for X in (S, T, Q, Z))
    r2 = gbr.reorder_gen_host(Sh, Th, Qh, Zh, sel, window=48, chain=20)
    assert np.array_equal(S1, Sh) and np.array_equal(T1, Th)
    assert np.array_equal(Q1, Qh) and np.array_equal(Z1, Zh)
    assert r1.m == r2.m and np.array_equal(r1.eigs, r2.eigs)


def test_rejected_swap_leaves_pair_unchanged(gbr):
    """The ill-conditioned 2x2|2x2 pair the oracle's pin rejects: the GPU
    rejects it too and leaves (S, T, Q, Z) untouched."""
    from tests.test_oracle_gen import ill_conditioned_pair
    S, T = ill_conditioned_pair()
    I4 = np.asfortranarray(np.eye(4))
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, I4, I4, [0, 0, 1, 1], window=8, chain=3)
    assert r.status == 1 and r.stats.rejected == 1
    r2, *_ = run_gpu(gbr, S, T, I4, I4, [0, 0, 1, 1], window=8, chain=3, sched="sequential")
    assert r2.status == 1
    assert np.array_equal(Sg, S) and np.array_equal(Tg, T)
    assert np.array_equal(Qg, I4) and np.array_equal(Zg, I4)


def test_invalid_pair_is_refused(gbr):
    S, T, Q, Z, sel = si.gen_problem(40, 2, reflectors=4)
    T[5, 2] = 1e-3   # below the diagonal of T
    with pytest.raises(gbr.GbrError) as ei:
        run_gpu(gbr, S, T, Q, Z, sel, allow_partial=False)
    assert ei.value.status == -2


def test_g4000_workload(gbr):
    """The n = 4000 pair workload: eigenvalue order against the input's
    blocks, exact structure, orthogonality and backward error of the whole
    result (the oracle takes minutes at this size)."""
    S, T, Q, Z, sel = si.gen_config("g4000")
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel)
    assert r.status == 0
    check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg)


@pytest.mark.parametrize("n,w,m", [(300, 64, 32), (515, 32, 12)])
def test_persistent_matches_sequential(gbr, n, w, m):
    """The persistent schedule (one launch, tasks ordered by dependences on
    exact rectangles of S/T, Q and Z) and the per-window launch pairs compute
    the same reordering up to the rounding of commuting updates."""
    S, T, Q, Z, sel = si.gen_problem(n, 31 + n, select_frac=0.45, reflectors=16)
    rp, Sp, Tp, Qp, Zp = run_gpu(gbr, S, T, Q, Z, sel, window=w, chain=m, sched="persistent")
    rs, Ss, Ts, Qs, Zs = run_gpu(gbr, S, T, Q, Z, sel, window=w, chain=m, sched="sequential")
    assert rp.status == rs.status == 0
    assert rp.stats.tasks > 0 and rs.stats.tasks == 0
    for a, b, ref in ((Sp, Ss, S), (Tp, Ts, T), (Qp, Qs, Q), (Zp, Zs, Z)):
        assert np.linalg.norm(a - b) <= 50 * n * EPS * np.linalg.norm(ref)
    check(S, T, Q, Z, sel, rp, Sp, Tp, Qp, Zp)


@pytest.mark.parametrize("prec", ["fma", "ozaki"])
def test_chunked_launches_match_one_launch(gbr, prec):
    """A pass of more than 1024 pair windows runs as three consecutive
    persistent launches, each planned while the previous one runs; together
    they keep the program order of one launch, so (S, T, Q, Z) come out
    bitwise as from a single traced (hence unchunked) launch."""
    n = 1200
    S, T, Q, Z, sel = si.gen_problem(n, 21, select_frac=0.5, reflectors=8)
    sub = np.append(np.diag(S, -1) != 0, False).astype(np.uint8)
    assert len(gbr.plan(sub, sel, 16, 6)[0]) >= 1024
    r1, S1, T1, Q1, Z1 = run_gpu(gbr, S, T, Q, Z, sel, window=16, chain=6, precision=prec)
    assert r1.status == 0
    check(S, T, Q, Z, sel, r1, S1, T1, Q1, Z1)
    r2, S2, T2, Q2, Z2 = run_gpu(gbr, S, T, Q, Z, sel, window=16, chain=6, precision=prec,
                                 timing=2)
    assert r2.status == 0 and r2.stats.tasks == r1.stats.tasks
    assert r1.stats.launches == r2.stats.launches + 2   # one pass, three launches
    for a, b in ((S1, S2), (T1, T2), (Q1, Q2), (Z1, Z2)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,n,w,m", [("n200", 200, 64, 32), ("ragged515", 515, 32, 12),
                                        ("g400", 400, 64, 32)])
def test_split_precision_updates(gbr, name, n, w, m):
    """Off-diagonal updates of S, T, Q, Z in emulated FP64 (7 digit slices of
    UQ and UZ, exact bf16 tensor-core products): the same parity bar as the
    DMMA path, and close to the DMMA result."""
    if name == "g400":
        S, T, Q, Z, sel = si.gen_config("g400")
    else:
        S, T, Q, Z, sel = si.gen_problem(n, n + 11, select_frac=0.4, reflectors=16)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    ro, So, To, Qo, Zo = run_gpu(gbr, S, T, Q, Z, sel, window=w, chain=m, precision="ozaki")
    assert ro.status == 0
    check(S, T, Q, Z, sel, ro, So, To, Qo, Zo, ref)
    rd, Sd, Td, Qd, Zd = run_gpu(gbr, S, T, Q, Z, sel, window=w, chain=m, precision="dmma")
    for a, b, x in ((So, Sd, S), (To, Td, T), (Qo, Qd, Q), (Zo, Zd, Z)):
        assert np.linalg.norm(a - b) <= 50 * n * EPS * np.linalg.norm(x)


def test_split_precision_g4000(gbr):
    S, T, Q, Z, sel = si.gen_config("g4000")
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel, precision="ozaki")
    assert r.status == 0
    check(S, T, Q, Z, sel, r, Sg, Tg, Qg, Zg)


@pytest.mark.parametrize("sched", ["persistent", "sequential"])
def test_rejections_clustered_nonnormal(gbr, sched):
    """Clustered generalized eigenvalues with strongly non-normal 2x2 parts
    (kappa = 1e6): some swaps are rejected and the pass loop re-plans around
    the stuck blocks.  Acceptance near the thresholds depends on rounding,
    so the oracle and the GPU may reject different swaps: both must return
    valid equivalences, the same eigenvalues as a set, and the same order
    up to the first block either one left stuck."""
    from scipy.optimize import linear_sum_assignment
    n = 300
    S, T, Q, Z, sel = si.gen_problem(n, 3, select_frac=0.5, clusters=True, spread=1e-6,
                                     kappa=1e6, reflectors=8)
    ref = oracle.gen_reorder(S, T, Q, Z, sel)
    r, Sg, Tg, Qg, Zg = run_gpu(gbr, S, T, Q, Z, sel, sched=sched)
    print(f"rejections: oracle {ref['nrej']}, gpu {r.status}")
    assert ref["status"] > 0 and r.status > 0
    assert is_gen_schur(Sg, Tg)
    assert orth_err(Qg) <= 50 * n * EPS and orth_err(Zg) <= 50 * n * EPS
    assert pair_residual(Q @ S @ Z.T, Q @ T @ Z.T, Sg, Tg, Qg, Zg) <= 50 * n * EPS
    a, b = gen_block_eigs(S, T), gen_block_eigs(Sg, Tg)
    cost = np.abs(a[:, None] - b[None, :])
    i, j = linear_sum_assignment(cost)
    assert cost[i, j].max() <= 1e-3   # attainable accuracy of these eigenvalues
    want, m = gen_expected_order(S, T, sel)
    got_o, got_g = ref["eigs"], b
    k = 0
    while k < m and abs(got_o[k] - want[k]) <= 1e-6 * max(1, abs(want[k])) and \
            abs(got_g[k] - want[k]) <= 1e-6 * max(1, abs(want[k])):
        k += 1
    assert k > 0
    assert match_eigs(got_g[:k], got_o[:k], 0) <= 1e-6
