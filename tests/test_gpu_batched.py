"""Batched reordering on the GPU (one task graph, one persistent launch from a
CUDA graph) against the CPU oracle, and against the single-problem entry
point: an instance's result must not depend on the batch around it."""
import numpy as np
import pytest

import oracle
import schur_inputs as si
from tests.helpers import EPS, block_eigs, expected_order, is_standard, orth_err, residual
from tests.test_gpu_parity import check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def instances(count, seed, nmin, nmax, q_every=1):
    out = []
    for i, (n, p, sd) in enumerate(si.batch_problems(count, seed, nmin, nmax)):
        S, Q, sel = si.reorder_problem(n, sd, select_frac=p, q="householder",
                                       reflectors=min(n, 64))
        out.append((S, Q if i % q_every == 0 else None, sel))
    return out


def to_dev(g, probs):
    Sd = [g.to_device(S) for S, _, _ in probs]
    Qd = [g.to_device(Q) if Q is not None else None for _, Q, _ in probs]
    return Sd, Qd


@pytest.mark.parametrize("w,m", [(128, 64), (64, 30), (32, 8)])
def test_batched_matches_oracle(gbr, w, m):
    probs = instances(24, 7, 1, 300, q_every=3)
    Sd, Qd = to_dev(gbr, probs)
    r = gbr.reorder_batched(Sd, Qd, [s for _, _, s in probs], window=w, chain=m)
    assert r.rc == 0 and np.all(r.status == 0)
    for i, (S, Q, sel) in enumerate(probs):
        ref = oracle.reorder(S, Q, sel)
        Sg = gbr.to_host(Sd[i])
        Qg = gbr.to_host(Qd[i]) if Qd[i] is not None else None

        class R:
            pass
        ri = R()
        ri.status, ri.m, ri.eigs = int(r.status[i]), int(r.m[i]), r.eigs[i]
        check(S, Q, sel, ri, Sg, Qg, ref)


@pytest.mark.parametrize("precision", ["dmma", "ozaki", "fma"])
def test_batched_equals_single_calls(gbr, precision):
    """Bitwise: every output element is computed by the same operations in
    the same order whatever the batch (tasks only regroup rows)."""
    probs = instances(16, 11, 20, 400)
    Sd, Qd = to_dev(gbr, probs)
    r = gbr.reorder_batched(Sd, Qd, [s for _, _, s in probs], window=96, chain=40,
                            precision=precision)
    assert r.rc == 0
    for i, (S, Q, sel) in enumerate(probs):
        S1, Q1 = gbr.to_device(S), gbr.to_device(Q)
        r1 = gbr.reorder(S1, Q1, sel, window=96, chain=40, precision=precision)
        assert r1.status == 0
        assert np.array_equal(gbr.to_host(S1), gbr.to_host(Sd[i]))
        assert np.array_equal(gbr.to_host(Q1), gbr.to_host(Qd[i]))
        assert np.array_equal(r1.eigs, r.eigs[i])


def test_graph_replay_and_plan_mismatch(gbr):
    probs = instances(12, 5, 40, 200)
    Sd, Qd = to_dev(gbr, probs)
    S0 = [s.clone() for s in Sd]
    Q0 = [q.clone() for q in Qd]
    with gbr.Batch(Sd, Qd, [s for _, _, s in probs], window=64, chain=24) as b:
        r1 = b.run()
        out1 = [gbr.to_host(s) for s in Sd]
        # replay on restored inputs: identical results
        for s, s0 in zip(Sd, S0):
            s.copy_(s0)
        for q, q0 in zip(Qd, Q0):
            q.copy_(q0)
        r2 = b.run()
        assert r1.rc == r2.rc == 0
        for s, o in zip(Sd, out1):
            assert np.array_equal(gbr.to_host(s), o)
        # the reordered forms have other 2x2 positions: the graph refuses them
        moved = [gbr.to_host(s) for s in Sd]
        with pytest.raises(gbr.GbrError) as ei:
            b.run()
        assert ei.value.status == gbr.ERR_PLAN_MISMATCH
        for s, o in zip(Sd, moved):
            assert np.array_equal(gbr.to_host(s), o)


def test_invalid_and_empty_instances(gbr):
    probs = instances(6, 9, 10, 80)
    S_bad = probs[2][0].copy(order="F")
    S_bad[5, 1] = 1e-3                       # below the subdiagonal
    probs[2] = (S_bad, probs[2][1], probs[2][2])
    probs.append((np.zeros((0, 0), order="F"), None, np.zeros(0, np.int32)))
    Sd, Qd = to_dev(gbr, probs)
    r = gbr.reorder_batched(Sd, Qd, [s for _, _, s in probs], window=64, chain=24)
    assert r.status[2] == -2
    assert np.array_equal(gbr.to_host(Sd[2]), S_bad)
    for i, (S, Q, sel) in enumerate(probs):
        if i == 2 or S.shape[0] == 0:
            continue
        assert r.status[i] == 0
        Sg = gbr.to_host(Sd[i])
        want, m = expected_order(S, sel)
        assert is_standard(Sg) and r.m[i] == m
        assert np.max(np.abs(block_eigs(Sg) - want) / np.maximum(np.abs(want), 1)) <= 1e-10


def test_batched_rejections_get_fixup_passes(gbr):
    """Clustered kappa = 1e6 instances reject swaps; their further passes run
    after the graph and the results stay exact similarities."""
    probs = [si.reorder_problem(n, 30 + n, select_frac=0.5, q="householder", reflectors=16,
                                clusters=True, spread=1e-6, kappa=1e6) for n in (120, 200)]
    probs += instances(4, 12, 30, 150)
    Sd, Qd = to_dev(gbr, probs)
    r = gbr.reorder_batched(Sd, Qd, [s for _, _, s in probs], window=64, chain=24)
    assert r.status[0] > 0 or r.status[1] > 0
    assert r.rc == int(np.sum(r.status > 0))
    for i, (S, Q, sel) in enumerate(probs):
        Sg, Qg = gbr.to_host(Sd[i]), gbr.to_host(Qd[i])
        n = S.shape[0]
        assert is_standard(Sg)
        assert residual(Q @ S @ Q.T, Sg, Qg) <= 50 * n * EPS
        assert orth_err(Qg) <= 50 * n * EPS


def test_autotuner_table_and_auto_options(gbr):
    tuned = gbr.autotune(64, 24)
    assert tuned == 2
    for n in (20, 50):
        w, m, t, ok = gbr.tune_get(n)
        assert ok and 4 <= w <= 128 and 1 <= m <= w - 2 and t in (64, 256)
    probs = instances(10, 21, 20, 64)
    Sd, Qd = to_dev(gbr, probs)
    r = gbr.reorder_batched(Sd, Qd, [s for _, _, s in probs], window=gbr.AUTO, chain=gbr.AUTO)
    assert r.rc == 0
    for i, (S, Q, sel) in enumerate(probs):
        ref = oracle.reorder(S, Q, sel)
        Sg, Qg = gbr.to_host(Sd[i]), gbr.to_host(Qd[i])

        class R:
            pass
        ri = R()
        ri.status, ri.m, ri.eigs = int(r.status[i]), int(r.m[i]), r.eigs[i]
        check(S, Q, sel, ri, Sg, Qg, ref)


def test_batched_trace(gbr):
    """opts.timing = 2 on a batch: the scheduler launch of the batch's graph
    records one timeline entry per task (all instances), readable with
    gbr_last_trace; every predecessor-free start is ordered sensibly."""
    probs = instances(12, 5, 40, 200)
    Sd, Qd = to_dev(gbr, probs)
    b = gbr.Batch(Sd, Qd, [s for _, _, s in probs], window=64, chain=30, timing=2)
    r = b.run()
    assert r.rc == 0
    tr = gbr.last_trace()
    assert len(tr) == r.stats.tasks > 0
    kind, win, _, _, _, take, start, end = tr.T
    assert set(np.unique(kind)) <= {0, 1, 2, 3}
    assert np.all(take <= start) and np.all(start <= end)
    assert int(np.sum(kind == 0)) == r.stats.windows
