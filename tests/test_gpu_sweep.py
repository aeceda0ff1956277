"""GPU bulge-chasing sweep (Section 3.2: one pipelined QR iteration by
overlapping 3x3 Householder reflectors, in windows with accumulated
transformations) through gbr_qr_sweep, against the CPU oracle.

The GPU applies the same reflectors in the same mathematical order (the
wavefront of a chase step equals the lowest-first sequence of the oracle),
so H and Q are compared element by element: H within 1e-10 ||H||, Q within
1e-8 (the chase amplifies rounding differences in the trailing entries
with the number of shifts; 1e-11 is typical at 32 shifts).  Plus exact
Hessenberg structure, orthogonality and backward error within 50 n eps.
"""
import numpy as np
import pytest

import oracle
import schur_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def gbr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1905_04975_gb300 as g
    g.load()
    return g


def run_gpu(g, H, Q, sh, **kw):
    Hd = g.to_device(H)
    Qd = g.to_device(Q) if Q is not None else None
    r = g.qr_sweep(Hd, Qd, sh, **kw)
    torch.cuda.synchronize()
    return r, g.to_host(Hd), (g.to_host(Qd) if Qd is not None else None)


def check(H, Q, sh, r, Hg, Qg, qtol=1e-8):
    n = H.shape[0]
    st, Ho, Qo = oracle.qr_sweep(H, Q, sh)
    assert st == 0 and r.status == 0
    assert np.all(np.tril(Hg, -2) == 0.0)
    assert np.max(np.abs(Hg - Ho)) <= 1e-10 * np.linalg.norm(H)
    if Qg is not None:
        assert np.max(np.abs(Qg - Qo)) <= qtol
        assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) <= 50 * n * EPS
        A = Q @ H @ Q.T
        assert np.linalg.norm(A - Qg @ Hg @ Qg.T) <= 50 * n * EPS * np.linalg.norm(A)


@pytest.mark.parametrize("n,ns,w,chain", [(3, 2, 96, 32), (4, 2, 96, 32), (7, 4, 8, 2),
                                          (10, 2, 96, 32), (50, 4, 16, 4), (97, 6, 24, 6),
                                          (200, 16, 48, 16), (300, 32, 96, 32),
                                          (515, 24, 64, 20)])
@pytest.mark.parametrize("sched", ["persistent", "sequential"])
def test_matches_oracle(gbr, n, ns, w, chain, sched):
    H, Q, sh = si.hessenberg_problem(n, n + ns, nshifts=ns, reflectors=8)
    r, Hg, Qg = run_gpu(gbr, H, Q, sh, window=w, chain=chain, sched=sched)
    check(H, Q, sh, r, Hg, Qg)
    if sched == "persistent" and r.stats.windows > 0:
        assert r.stats.tasks > 0


def test_h400_workload_and_without_q(gbr):
    H, Q, sh = si.sweep_config("h400")
    r, Hg, Qg = run_gpu(gbr, H, Q, sh, sched="sequential")
    check(H, Q, sh, r, Hg, Qg)
    r2, Hg2, _ = run_gpu(gbr, H, None, sh, sched="sequential")
    assert np.array_equal(Hg, Hg2)


def test_h4000_workload(gbr):
    """The n = 4000 sweep with 64 shifts (persistent schedule): element-wise
    against the oracle (which takes a few seconds here), structure,
    orthogonality and backward error."""
    H, Q, sh = si.sweep_config("h4000")
    r, Hg, Qg = run_gpu(gbr, H, Q, sh)
    check(H, Q, sh, r, Hg, Qg)


def test_exact_shifts_deflate(gbr):
    """Shifts = a conjugate pair of eigenvalues of H: the pair splits off at
    the bottom (n = 30, three windows of 16; larger random Hessenberg
    matrices have eigenvalues too ill-conditioned for this)."""
    n = 30
    H, _, _ = si.hessenberg_problem(n, 3, nshifts=2, reflectors=4)
    w = np.linalg.eigvals(H)
    c = [x for x in w if x.imag > 1e-3][0]
    r, Hg, _ = run_gpu(gbr, H, None, [c, np.conj(c)], window=16, chain=2, sched="sequential")
    assert r.stats.windows >= 2
    assert abs(Hg[n - 2, n - 3]) <= 1e-10 * np.linalg.norm(H)
    assert abs(H[n - 2, n - 3]) > 1e-3


def test_not_hessenberg_is_refused(gbr):
    H, Q, sh = si.hessenberg_problem(40, 1, nshifts=4)
    H[10, 3] = 1.0
    with pytest.raises(gbr.GbrError) as ei:
        run_gpu(gbr, H, Q, sh, sched="sequential")
    assert ei.value.status == -2


def test_reducible_hessenberg(gbr):
    """A zero subdiagonal entry stops the bulges that reach it (their
    reflectors become the identity there); GPU and oracle agree."""
    n = 120
    H, Q, sh = si.hessenberg_problem(n, 21, nshifts=8, reflectors=4)
    H[60, 59] = 0.0
    r, Hg, Qg = run_gpu(gbr, H, Q, sh, window=32, chain=4)
    check(H, Q, sh, r, Hg, Qg)


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_smallest_sizes_many_shifts(gbr, n):
    """More bulges than the matrix can hold at once: the chains still run to
    the end on both schedules."""
    H, Q, sh = si.hessenberg_problem(n, 40 + n, nshifts=8, reflectors=2)
    for sched in ("persistent", "sequential"):
        r, Hg, Qg = run_gpu(gbr, H, Q, sh, window=8, chain=2, sched=sched)
        check(H, Q, sh, r, Hg, Qg)
