"""Host-side window planner (gbr_plan): windows never cut a 2x2 block, stay
within the window size, and -- replayed as stable partitions of the blocks
they cover -- produce exactly the stable partition the reordering defines.
The replay below is plain permutation bookkeeping, independent of the
planner's C++ code."""
import numpy as np
import pytest

import paper_1905_04975_gb300 as g
import schur_inputs as si
from paper_1905_04975_gb300 import build as gbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    return g.load()


def layout(sizes, sel_blocks):
    """List of blocks (size, selected) in diagonal order."""
    return [(int(s), bool(v)) for s, v in zip(sizes, sel_blocks)]


def replay(blocks, windows):
    """Apply each window as the stable partition of the blocks it covers."""
    blocks = list(blocks)
    for s, e in windows:
        starts = np.concatenate([[0], np.cumsum([b[0] for b in blocks])])
        i0 = int(np.searchsorted(starts, s))
        i1 = int(np.searchsorted(starts, e))
        assert starts[i0] == s, f"window start {s} cuts a 2x2 block"
        assert starts[i1] == e, f"window end {e} cuts a 2x2 block"
        seg = blocks[i0:i1]
        blocks[i0:i1] = [b for b in seg if b[1]] + [b for b in seg if not b[1]]
    return blocks


def problem(n, seed, frac):
    rng = np.random.default_rng(seed)
    sizes = si.block_sizes(n, rng)
    sel = si.selection(sizes, frac, rng)
    sub = np.zeros(n, np.uint8)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    selb = []
    for st, sz in zip(starts, sizes):
        if sz == 2:
            sub[st] = 1
        selb.append(bool(sel[st]))
    return sizes, sel, sub, selb


@pytest.mark.parametrize("n,seed,frac,w,m", [
    (400, 0, 0.3, 128, 64), (4000, 0, 0.35, 128, 64), (1000, 1, 0.5, 64, 30),
    (257, 2, 0.2, 16, 6), (130, 3, 0.9, 32, 10), (50, 4, 0.05, 8, 3), (3, 5, 0.5, 4, 2),
    (1, 6, 1.0, 4, 1), (4000, 0, 0.35, 256, 128), (1000, 1, 0.5, 200, 150),
    (600, 2, 0.6, 256, 254)])
def test_plan_is_the_stable_partition(n, seed, frac, w, m):
    sizes, sel, sub, selb = problem(n, seed, frac)
    W, chains, flops = g.plan(sub, sel, w, m)
    assert np.all(W[:, 1] - W[:, 0] <= w) and np.all(W[:, 1] > W[:, 0])
    assert np.all(W[:, 0] >= 0) and np.all(W[:, 1] <= n)
    blocks = layout(sizes, selb)
    final = replay(blocks, W)
    want = [b for b in blocks if b[1]] + [b for b in blocks if not b[1]]
    assert final == want
    # flop count of the off-diagonal updates (with Q)
    ww = (W[:, 1] - W[:, 0]).astype(float)
    assert flops == pytest.approx(float(np.sum(2 * ww * ww * ((n - W[:, 1]) + W[:, 0] + n))))


def test_plan_edge_cases():
    assert g.plan(np.zeros(5, np.uint8), np.zeros(5, np.int32))[0].shape == (0, 2)
    assert g.plan(np.zeros(5, np.uint8), np.ones(5, np.int32))[0].shape == (0, 2)
    # a selected last block needs windows; a selected first block none
    sub = np.zeros(6, np.uint8)
    assert len(g.plan(sub, np.array([1, 0, 0, 0, 0, 0], np.int32), 4, 2)[0]) == 0
    W = g.plan(sub, np.array([0, 0, 0, 0, 0, 1], np.int32), 4, 2)[0]
    assert len(W) >= 2 and W[-1, 0] == 0
    with pytest.raises(g.GbrError):
        g.plan(sub, np.zeros(6, np.int32), 257, 64)
    with pytest.raises(g.GbrError):
        g.plan(sub, np.zeros(6, np.int32), 256, 255)
