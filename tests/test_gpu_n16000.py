"""The clustered n = 16000 workload at full size, every precision of the
off-diagonal updates (FP64 DMMA, FP64 FMA tiles and split precision),
through the C ABI.

This is the configuration with the largest update tiles (1024-row far
tiles) and the largest task graph (about 347 K tasks).  The oracle needs
hours at this size, so the result is checked against what holds at any
size (Eq. 7):
  * S is in standard real Schur form (exact zeros below the
    quasi-diagonal, standardized 2x2 blocks);
  * the eigenvalues on its diagonal are the stable partition of the input
    eigenvalues (selected first, relative order kept in both sets), to
    1e-10 relative -- clusters of spread 1e-6 make a misordered pair show
    up as an error near 1e-6;
  * ||Q^T Q - I||_F <= 50 n eps and ||A - Q S Q^T||_F / ||A||_F <= 50 n eps
    with A = Q0 S0 Q0^T, computed on the GPU with FP64 matrix products
    (||A - Q S Q^T||_F = ||S0 - W S W^T||_F with W = Q0^T Q, up to the
    rounding of the input's orthogonality);
  * the rejected swaps are counted and reported; with rejections the order
    is compared before the first stuck block only.
"""
import numpy as np
import pytest

import schur_inputs as si
from tests.helpers import EPS, block_eigs, expected_order, is_standard

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="module")
def workload():
    S, Q, sel = si.config("n16000c")
    want, m = expected_order(S, sel)
    return S, Q, sel, want, m


def fro(X):
    return float(torch.linalg.norm(X).item())


@pytest.mark.parametrize("prec", ["dmma", "ozaki", "fma"])
def test_n16000c_full_size(gbr, workload, prec):
    S_np, Q_np, sel, want, m = workload
    n = S_np.shape[0]
    g = gbr
    Sd, Qd = g.to_device(S_np), g.to_device(Q_np)
    r = g.reorder(Sd, Qd, sel, precision=prec, window=128, chain=64)
    torch.cuda.synchronize()
    print(f"n16000c {prec}: status {r.status}, rejected {r.stats.rejected}, "
          f"windows {r.stats.windows}, tasks {r.stats.tasks}, swaps {r.stats.swaps}")
    assert r.status >= 0 and r.m == m
    assert r.stats.tasks > 300000          # the n = 16000 task graph ran
    Sg = g.to_host(Sd)
    assert is_standard(Sg)
    got = block_eigs(Sg)
    assert np.max(np.abs(r.eigs - got) / np.maximum(np.abs(got), 1.0)) <= 1e-14
    dev = np.abs(got - want) / np.maximum(np.abs(want), 1.0)
    if r.status == 0:
        assert float(np.max(dev)) <= 1e-10
    else:
        k = int(np.argmax(dev > 1e-10)) if np.any(dev > 1e-10) else n
        print(f"order agrees on the first {k} positions")
        assert k > 0
    del Sg
    # orthogonality and residual: FP64 products on the GPU
    bound = 50 * n * EPS
    Qc = Qd.contiguous()
    QtQ = Qc.T @ Qc
    QtQ.diagonal().sub_(1.0)
    orth = fro(QtQ)
    del QtQ
    S0 = g.to_device(S_np).contiguous()
    Q0 = g.to_device(Q_np).contiguous()
    W = Q0.T @ Qc
    del Qc, Q0
    E = W @ (Sd.contiguous() @ W.T)
    E.sub_(S0)
    res = fro(E) / fro(S0)
    print(f"n16000c {prec}: orthogonality {orth:.3e}, residual {res:.3e}, bound {bound:.3e}")
    assert orth <= bound
    assert res <= bound
