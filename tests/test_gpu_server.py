"""The reordering server (continuous batching) on the GPU: every request's
result equals the same request run alone, admission respects the memory
cap, requests submitted while others run are launched alongside them, and
failures stay per request."""
import time

import numpy as np
import pytest

import schur_inputs as si
from tests.helpers import EPS, expected_order, is_standard, orth_err, residual, block_eigs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def stream_of(count, seed, nmin, nmax):
    out = []
    for _, n, p, sd in si.request_stream(count, seed, nmin, nmax):
        S, Q, sel = si.reorder_problem(n, sd, select_frac=p, q="householder",
                                       reflectors=min(n, 64))
        out.append((S, Q, sel))
    return out


def alone(g, S, Q, sel, **kw):
    Sd, Qd = g.to_device(S), g.to_device(Q)
    r = g.reorder(Sd, Qd, sel, **kw)
    return r, g.to_host(Sd), g.to_host(Qd)


@pytest.mark.parametrize("precision", ["dmma", "ozaki", "fma"])
def test_mix_equals_alone(gbr, precision):
    probs = stream_of(30, 1, 16, 900)
    with gbr.Server(window=128, chain=64, precision=precision) as srv:
        work = [(S.copy(order="F"), Q.copy(order="F"), sel) for S, Q, sel in probs]
        tickets = [srv.submit(S, Q, sel) for S, Q, sel in work]
        res = [srv.wait(t, 120000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert st["mean_inflight"] > 1    # requests shared the device
    for (S, Q, sel), (Sw, Qw, _), r in zip(probs, work, res):
        assert r.status == 0
        ra, Sa, Qa = alone(gbr, S, Q, sel, window=128, chain=64, precision=precision)
        assert np.array_equal(Sw, Sa) and np.array_equal(Qw, Qa)
        assert np.array_equal(r.eigs, ra.eigs) and r.m == ra.m


def test_admission_cap_and_stats(gbr):
    probs = stream_of(24, 2, 200, 700)
    big = max(S.shape[0] for S, _, _ in probs)
    cap = 3 * (2 * big * big * 8) + (64 << 20)
    with gbr.Server(mem_cap_bytes=cap) as srv:
        work = [(S.copy(order="F"), Q.copy(order="F"), sel) for S, Q, sel in probs]
        tickets = [srv.submit(S, Q, sel) for S, Q, sel in work]
        res = [srv.wait(t, 120000) for t in tickets]
        st = srv.stats()
    assert all(r is not None and r.status == 0 for r in res)
    assert 0 < st["peak_mem_bytes"] <= cap
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["req_per_s"] > 0 and st["eigs_per_s"] > 0
    for (S, Q, sel), (Sw, Qw, _) in zip(probs, work):
        n = S.shape[0]
        want, m = expected_order(S, sel)
        assert is_standard(Sw)
        assert np.max(np.abs(block_eigs(Sw) - want) / np.maximum(np.abs(want), 1)) <= 1e-10
        assert residual(Q @ S @ Q.T, Sw, Qw) <= 50 * n * EPS
        assert orth_err(Qw) <= 50 * n * EPS


def test_small_requests_run_beside_a_large_one(gbr):
    """Continuous batching: requests that arrive while a large one is on the
    GPU are admitted at once, their tasks enter the ring between its tasks,
    and they finish before it."""
    S, Q, sel = si.reorder_problem(6000, 5, select_frac=0.4, q="householder")
    small = stream_of(6, 3, 40, 120)
    with gbr.Server() as srv:
        tb = srv.submit(S, Q, sel, eigs=False)
        time.sleep(0.02)
        ts = [srv.submit(s.copy(order="F"), q.copy(order="F"), sl) for s, q, sl in small]
        done_small = [srv.wait(t, 60000) for t in ts]
        big_pending = srv.poll(tb) is None
        rb = srv.wait(tb, 120000)
    assert all(r.status == 0 for r in done_small)
    assert rb.status == 0
    assert big_pending


def test_invalid_oversized_and_rejecting_requests(gbr):
    ok = stream_of(3, 4, 30, 80)
    bad = ok[0][0].copy(order="F")
    bad[4, 1] = 0.5                      # below the subdiagonal
    rej = si.reorder_problem(150, 44, select_frac=0.5, q="householder", reflectors=16,
                             clusters=True, spread=1e-6, kappa=1e6)
    with gbr.Server(mem_cap_bytes=64 << 20) as srv:
        with pytest.raises(gbr.GbrError) as ei:
            srv.submit(np.zeros((3000, 3000), order="F"), np.eye(3000, order="F"),
                       np.ones(3000, np.int32))
        assert ei.value.status == gbr.ERR_NOMEM
        tb = srv.submit(bad, ok[0][1].copy(order="F"), ok[0][2])
        Sr, Qr = rej[0].copy(order="F"), rej[1].copy(order="F")
        tr = srv.submit(Sr, Qr, rej[2])
        good = [(S.copy(order="F"), Q.copy(order="F"), s) for S, Q, s in ok[1:]]
        tg = [srv.submit(*x) for x in good]
        rbad = srv.wait(tb, 60000)
        rrej = srv.wait(tr, 60000)
        rg = [srv.wait(t, 60000) for t in tg]
    assert rbad.status == -2
    assert rrej.status > 0
    n = rej[0].shape[0]
    assert is_standard(Sr)
    assert residual(rej[1] @ rej[0] @ rej[1].T, Sr, Qr) <= 50 * n * EPS
    assert all(r.status == 0 for r in rg)
