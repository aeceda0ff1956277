"""gbr_reorder_noalloc: the reordering entry point for callers that cannot
allocate device memory (programs whose device memory is all handed out by
their own arena, or that must not have a cudaMalloc synchronize the device
in the middle of their work).  Its scratch is a fixed device array in the
library image.  Its results must match gbr_reorder's, call after call: the
shared scratch keeps the previous call's contents, so a second call must
start from a clean state.  And it must really allocate nothing: in a fresh
process whose first library call is this one, the library's pool stays
empty and the device's free memory does not change across a call.

This file is collected last so that, in a run that stops at the first
failure, every other test has already run.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import schur_inputs as si
from tests.helpers import EPS, expected_order, match_eigs, orth_err, residual

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def run(g, fn, S, Q, sel, **kw):
    Sd, Qd = g.to_device(S), g.to_device(Q)
    r = fn(Sd, Qd, sel, **kw)
    torch.cuda.synchronize()
    return r, g.to_host(Sd), g.to_host(Qd)


@pytest.mark.parametrize("case", ["n400", "ragged700"])
def test_noalloc_matches_reorder_twice(g, case):
    if case == "n400":
        S, Q, sel = si.config("n400")
        kw = {}
    else:
        S, Q, sel = si.reorder_problem(700, 77, select_frac=0.4, q="householder")
        kw = dict(window=64, chain=30)
    n = S.shape[0]
    A = Q @ S @ Q.T
    ref, Sr, Qr = run(g, g.reorder, S, Q, sel, **kw)
    assert ref.status == 0
    want, m = expected_order(S, sel)
    for call in range(2):
        r, Sn, Qn = run(g, g.reorder_noalloc, S, Q, sel, **kw)
        assert r.status == 0 and r.m == ref.m == m
        # same results as the allocating entry point, within the tests' tolerances
        assert match_eigs(r.eigs, ref.eigs, 0) <= 1e-10
        assert np.linalg.norm(Sn - Sr) <= 50 * n * EPS * np.linalg.norm(S)
        assert np.linalg.norm(Qn - Qr) <= 50 * n * EPS * np.sqrt(n)
        assert match_eigs(r.eigs, want, 0) <= 1e-10
        assert orth_err(Qn) <= 50 * n * EPS
        assert residual(A, Sn, Qn) <= 50 * n * EPS
        assert r.stats.windows == ref.stats.windows


def test_capturing_stream_is_refused(g):
    """The entry points synchronize their stream, which a CUDA graph capture
    refuses: on a capturing stream they return ERR_CAPTURING before they
    enqueue anything.  S and Q stay untouched and the capture stays valid
    (the graph captured around the calls replays and computes its own
    work)."""
    S, Q, sel = si.reorder_problem(96, 5, select_frac=0.4, q="householder")
    Sd, Qd = g.to_device(S), g.to_device(Q)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
        x.add_(1.0)
        for fn in (g.reorder_noalloc, g.reorder):
            try:
                fn(Sd, Qd, sel)
                codes.append(0)
            except g.GbrError as e:
                codes.append(e.status)
        x.mul_(3.0)
    assert codes == [g.ERR_CAPTURING, g.ERR_CAPTURING]
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.full_like(x, 3.0))
    assert np.array_equal(g.to_host(Sd), S) and np.array_equal(g.to_host(Qd), Q)


def test_noalloc_rejects_oversized(g):
    lib = g.load()
    n = g.NOALLOC_MAX_N + 1
    sel = np.zeros(n, np.int32)
    dummy = ctypes.c_void_p(0x1000)   # never touched: the size check comes first
    rc = lib.gbr_reorder_noalloc(n, dummy, n, None, n,
                                 sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 None, None, None, None, None, None)
    assert rc == g.ERR_NOALLOC_LIMIT
    assert b"GBR_NOALLOC_MAX_N" in lib.gbr_status_string(rc)


_FRESH = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_1905_04975_gb300 as g
import schur_inputs as si
lib = g.load()
torch.cuda.set_device(0)
S, Q, sel = si.reorder_problem(500, 5, select_frac=0.4, q="householder")
Sd, Qd = g.to_device(S), g.to_device(Q)          # the caller's buffers
S0, Q0 = Sd.clone(), Qd.clone()
torch.cuda.synchronize()
out = []
for call in range(3):
    Sd.copy_(S0)
    Qd.copy_(Q0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    r = g.reorder_noalloc(Sd, Qd, sel)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    out.append([int(r.status), int(lib.gbr_pool_bytes()), int(free0), int(free1),
                float(r.eigs[0].real)])
print(json.dumps(out))
"""


def test_noalloc_allocates_nothing_in_a_fresh_process(g):
    """A process whose first library call is gbr_reorder_noalloc: the pool
    stays empty, and after the first call (which may load the library's
    module, array included, into the context) the device's free memory is
    the same before and after each call."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    calls = json.loads(p.stdout.strip().splitlines()[-1])
    assert len(calls) == 3
    for status, pool, free0, free1, eig0 in calls:
        assert status == 0
        assert pool == 0
    for status, pool, free0, free1, eig0 in calls[1:]:
        assert free1 == free0
    assert calls[0][4] == calls[1][4] == calls[2][4]
