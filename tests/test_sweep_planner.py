"""Host logic of the bulge-chasing sweep (runs without a GPU): the window
plan exported as gbr_plan_sweep keeps every active bulge inside its window,
covers every chase step of every chain exactly once, and a numpy replay of
the windowed chase with accumulated U (the GPU's structure: per window, the
chase steps on the window only, then U applied to the rows to the right,
the columns above and Q) reproduces the oracle."""
import numpy as np
import pytest

import oracle
import schur_inputs as si
import paper_1905_04975_gb300 as g
from paper_1905_04975_gb300 import build as gbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    return g.load()


def check_plan(n, nshifts, window, chain):
    P = g.plan_sweep(n, nshifts, window, chain)
    nb_total = nshifts // 2
    if n < 3 or nb_total == 0:
        assert len(P) == 0
        return P
    w = min(window, 96)
    nbc = max(1, min(chain // 2, w // 6))
    chains = {}
    for s, e, t0, t1, b0, nb in P:
        assert 0 <= s < e <= n and e - s <= w
        assert 1 <= nb <= nbc and b0 % nbc == 0
        chains.setdefault(b0, []).append((s, e, t0, t1, nb))
    assert sorted(chains) == list(range(0, nb_total, nbc))
    for b0, ws in chains.items():
        nb = ws[0][4]
        t_end = (n - 3) + 3 * (nb - 1) + 2
        assert ws[0][2] == 0 and ws[-1][3] == t_end
        for (a, b) in zip(ws, ws[1:]):
            assert a[3] == b[2]                      # contiguous step ranges
        for s, e, t0, t1, _ in ws:
            assert t1 > t0
            for tau in range(t0, t1):
                for j in range(nb):
                    k = tau - 3 * j - 1
                    if k < -1 or k > n - 3:
                        continue
                    if k == -1:
                        assert s == 0
                    else:
                        assert s <= k
                        length = 3 if k + 3 <= n - 1 else 2
                        assert k + length <= e - 1
                        assert k + 4 <= e - 1 or e == n
    return P


@pytest.mark.parametrize("n", [3, 4, 5, 9, 40, 97, 300, 1001])
@pytest.mark.parametrize("nshifts,window,chain", [(2, 8, 2), (8, 8, 2), (8, 16, 4), (16, 64, 16),
                                                  (24, 96, 32), (64, 64, 16), (6, 24, 6)])
def test_plan_invariants(n, nshifts, window, chain):
    check_plan(n, nshifts, window, chain)


def test_plan_arguments():
    assert g.load().gbr_plan_sweep(-1, 2, 64, 16, None, 0) == -1
    assert g.load().gbr_plan_sweep(10, 3, 64, 16, None, 0) == -1
    assert g.load().gbr_plan_sweep(10, 2, 2, 16, None, 0) == -10
    assert g.load().gbr_plan_sweep(10, 2, 64, 0, None, 0) == -10
    assert len(check_plan(2, 8, 64, 16)) == 0


def refl(x):
    x = np.asarray(x, float)
    v = np.zeros(len(x))
    v[0] = 1.0
    sig = float(np.sum(x[1:] ** 2))
    if sig == 0.0:
        return v, 0.0, x[0]
    nrm = np.sqrt(x[0] ** 2 + sig)
    b = -nrm if x[0] >= 0 else nrm
    v[1:] = x[1:] / (x[0] - b)
    return v, (b - x[0]) / b, b


def replay(H, Q, shifts, P):
    """The windowed chase of the plan in numpy (one reflector per active
    bulge per step, all reflectors of a step first, then the left products,
    then the right ones; U accumulated per window and applied after it)."""
    H, Q = H.copy(), Q.copy()
    n = H.shape[0]
    sp = [((shifts[2 * j] + shifts[2 * j + 1]).real, (shifts[2 * j] * shifts[2 * j + 1]).real)
          for j in range(len(shifts) // 2)]
    for s, e, t0, t1, b0, nb in P:
        ww = e - s
        Hs = H[s:e, s:e].copy()
        U = np.eye(ww)
        for tau in range(t0, t1):
            refls = []
            for j in range(nb):
                k = tau - 3 * j - 1
                if k < -1 or k > n - 3:
                    continue
                if k < 0:
                    ss, pp = sp[b0 + j]
                    x = [Hs[0, 0] ** 2 + Hs[0, 1] * Hs[1, 0] - ss * Hs[0, 0] + pp,
                         Hs[1, 0] * (Hs[0, 0] + Hs[1, 1] - ss), Hs[1, 0] * Hs[2, 1]]
                    kl, ln = -1, 3
                else:
                    kl = k - s
                    ln = 3 if k + 3 <= n - 1 else 2
                    x = Hs[kl + 1:kl + 1 + ln, kl]
                refls.append((kl, ln) + refl(x))
            for kl, ln, v, t, b in refls:
                c0, r = max(kl, 0), slice(kl + 1, kl + 1 + ln)
                Hs[r, c0:] -= t * np.outer(v, v @ Hs[r, c0:])
                if kl >= 0:
                    Hs[kl + 1, kl] = b
                    Hs[kl + 2:kl + 1 + ln, kl] = 0.0
            for kl, ln, v, t, b in refls:
                c = slice(kl + 1, kl + 1 + ln)
                rend = min(kl + 5, ww)
                Hs[:rend, c] -= t * np.outer(Hs[:rend, c] @ v, v)
                U[:, c] -= t * np.outer(U[:, c] @ v, v)
        H[s:e, s:e] = Hs
        H[s:e, e:] = U.T @ H[s:e, e:]
        H[:s, s:e] = H[:s, s:e] @ U
        Q[:, s:e] = Q[:, s:e] @ U
    return H, Q


@pytest.mark.parametrize("n,ns,window,chain", [(10, 2, 96, 32), (50, 4, 16, 4), (97, 6, 24, 6),
                                                (200, 16, 48, 16), (300, 32, 64, 16)])
def test_windowed_replay_matches_oracle(n, ns, window, chain):
    H, Q, sh = si.hessenberg_problem(n, n + ns, nshifts=ns, reflectors=4)
    P = check_plan(n, ns, window, chain)
    Hr, Qr = replay(H, Q, sh, P)
    st, Ho, Qo = oracle.qr_sweep(H, Q, sh)
    assert st == 0
    assert np.all(np.tril(Hr, -2) == 0.0)
    assert np.max(np.abs(Hr - Ho)) <= 1e-10 * np.linalg.norm(H)
    assert np.max(np.abs(Qr - Qo)) <= 1e-8


def test_plan_random_shapes():
    """Seeded random shapes (n, shifts, window >= 8, chain): the invariants
    hold and every chain makes progress; a window below 8 is refused."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        n = int(rng.choice([3, 4, 5, 6, 7, 8, 10, 13, 20, 33, 64, 65, 96, 97, 128, 200, 257]))
        check_plan(n, 2 * int(rng.integers(1, 41)), int(rng.integers(8, 129)),
                   int(rng.integers(1, 81)))
    for w in (4, 5, 7):
        assert g.load().gbr_plan_sweep(100, 8, w, 4, None, 0) == -10
