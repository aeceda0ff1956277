"""Seeded synthetic inputs for Schur-form eigenvalue reordering.

This module builds the test and benchmark inputs: a real Schur form S in
standard form (Eq. 4: upper quasi-triangular, 1x1 and 2x2 diagonal blocks),
an orthogonal factor Q, and a per-eigenvalue selection vector. It holds
none of the reordering arithmetic; the CPU oracle and the GPU library both
consume what it returns, and neither is imported here.

Workload recipe (the paper prints no reordering workload, so these shapes
are this project's synthetic stand-in):

* diagonal positions: round(0.6 n) in 1x1 blocks, the rest in 2x2 blocks
  (one more 1x1 if the remainder is odd); block order shuffled by the seed;
* 1x1 eigenvalues ~ N(0,1); 2x2 blocks [[a, b], [c, a]] with a ~ N(0,1),
  |b|, |c| ~ U(0.1, 2), sign(b) random and sign(c) = -sign(b), so bc < 0;
* strict upper triangle ~ N(0,1) (outside the 2x2 blocks);
* optional clustering: 12 real and 8 complex centres, each block being a
  centre perturbed by `spread` (additively for a, relatively for b and c);
* Q = identity, or the product H_1 ... H_k of k seeded Householder
  reflectors H_i = I - 2 v v^T / v^T v with v ~ N(0,1)^n;
* selection: blocks in seeded random order are selected until the selected
  eigenvalue count reaches round(p n); a 2x2 block (a conjugate pair) is
  always selected whole;
* serving requests: an independent form of order n per request from this
  generator (serve_problem, Q of 8 seeded reflectors), made when the
  request is about to arrive; or (serve_request, for the CPU sample of the
  reference arm) a principal diagonal block S[k:k+n, k:k+n] of one seeded
  base form cut at block boundaries, at a seeded offset k.

Generalized real Schur form (S, T) (the pair case of Eq. 7):

* block sizes and selection as above;
* T upper triangular: diagonal ~ U(0.5, 2), strict upper triangle ~ N(0,1);
* a 1x1 block of S is lambda t_jj with lambda ~ N(0,1) (so the generalized
  eigenvalue is lambda); a 2x2 block of S is T_b M with T_b the 2x2 diagonal
  block of T and M = [[a, b], [c, a]] drawn as for the standard form, so the
  pair's eigenvalues are a +- i sqrt(-bc); strict upper triangle of S
  (outside the blocks) ~ N(0,1);
* Q and Z: products of seeded Householder reflectors (as Q above), drawn
  one after the other from the same generator.

Bulge-chasing sweep (Schur reduction):

* H upper Hessenberg: entries on and above the subdiagonal ~ N(0,1);
* Q: product of seeded Householder reflectors (as above);
* shifts: s pairs, alternately a complex-conjugate pair a +- i b
  (a ~ N(0,1), b ~ U(0.1, 1)) and two real shifts ~ N(0,1).

All matrices are float64 in column-major (Fortran) order.
"""
from __future__ import annotations

import numpy as np

__all__ = ["block_sizes", "schur_form", "householder_q", "selection",
           "reorder_problem", "batch_problems", "request_stream", "serve_base",
           "serve_request", "serve_problem", "gen_schur_pair", "gen_problem", "gen_config",
           "hessenberg_problem", "sweep_config"]


def block_sizes(n: int, rng: np.random.Generator, frac_1x1: float = 0.6) -> np.ndarray:
    """Shuffled list of diagonal block sizes (1 or 2) covering n positions."""
    if n <= 0:
        return np.zeros(0, dtype=np.int64)
    n1 = int(round(frac_1x1 * n))
    n1 = min(max(n1, 0), n)
    n2 = n - n1
    if n2 % 2:
        n1 += 1
        n2 -= 1
    sizes = np.array([1] * n1 + [2] * (n2 // 2), dtype=np.int64)
    return sizes[rng.permutation(sizes.size)]


def schur_form(n: int, rng: np.random.Generator, *, frac_1x1: float = 0.6,
               clusters: bool = False, spread: float = 1e-6, kappa: float = 1.0,
               order: str = "F"):
    """Random standard real Schur form. Returns (S, sizes); S in the given
    memory order (the values do not depend on it).

    kappa > 1 makes the 2x2 blocks non-normal (|b| scaled by kappa, |c| by
    1/kappa, eigenvalues' imaginary parts unchanged); with clustered,
    nearly equal eigenvalues this is what makes block swaps ill-conditioned
    enough to be rejected."""
    sizes = block_sizes(n, rng, frac_1x1)
    S = np.zeros((n, n), dtype=np.float64, order=order)
    if n == 0:
        return S, sizes
    # strict upper triangle ~ N(0,1)
    upper = rng.standard_normal((n, n))
    if order == "C":
        S = np.triu(upper, k=1)
    else:
        S[:] = np.triu(upper, k=1)
    del upper
    nb1 = int(np.sum(sizes == 1))
    nb2 = int(np.sum(sizes == 2))
    if clusters:
        rc = rng.standard_normal(12)
        ca = rng.standard_normal(8)
        cb = rng.uniform(0.1, 2.0, 8) * rng.choice([-1.0, 1.0], 8)
        cc = -np.sign(cb) * rng.uniform(0.1, 2.0, 8)
        pick1 = rng.integers(0, 12, nb1)
        lam = rc[pick1] + spread * rng.standard_normal(nb1)
        pick2 = rng.integers(0, 8, nb2)
        a = ca[pick2] + spread * rng.standard_normal(nb2)
        b = cb[pick2] * (1.0 + spread * rng.standard_normal(nb2))
        c = cc[pick2] * (1.0 + spread * rng.standard_normal(nb2))
    else:
        lam = rng.standard_normal(nb1)
        a = rng.standard_normal(nb2)
        b = rng.uniform(0.1, 2.0, nb2) * rng.choice([-1.0, 1.0], nb2)
        c = -np.sign(b) * rng.uniform(0.1, 2.0, nb2)
    if kappa != 1.0:
        b = b * kappa
        c = c / kappa
    i1 = i2 = 0
    pos = 0
    for sz in sizes:
        if sz == 1:
            S[pos, pos] = lam[i1]
            i1 += 1
        else:
            S[pos, pos] = a[i2]
            S[pos + 1, pos + 1] = a[i2]
            S[pos, pos + 1] = b[i2]
            S[pos + 1, pos] = c[i2]
            i2 += 1
        pos += int(sz)
    return S, sizes


def householder_q(n: int, rng: np.random.Generator, k: int = 64,
                  order: str = "F") -> np.ndarray:
    """Q = H_1 H_2 ... H_k, H_i = I - 2 v_i v_i^T / (v_i^T v_i), v_i ~ N(0,1)^n.

    Formed in compact WY form, Q = I - V T V^T with T upper triangular, so
    that large n costs one matrix product.  Memory order as given (the
    values do not depend on it).
    """
    k = min(k, n)
    Q = np.zeros((n, n), dtype=np.float64, order=order)
    if n == 0:
        return Q
    V = rng.standard_normal((n, k))
    tau = 2.0 / np.einsum("ij,ij->j", V, V)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = tau[i]
        if i:
            T[:i, i] = -tau[i] * (T[:i, :i] @ (V[:, :i].T @ V[:, i]))
    if order == "C":
        Q = -(V @ T) @ V.T
    else:
        Q[:] = -(V @ T) @ V.T
    Q[np.diag_indices(n)] += 1.0
    return Q


def selection(sizes: np.ndarray, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Per-eigenvalue selection (int32, 0/1); 2x2 blocks are selected whole."""
    n = int(np.sum(sizes))
    sel = np.zeros(n, dtype=np.int32)
    if n == 0:
        return sel
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    target = int(round(frac * n))
    count = 0
    for b in rng.permutation(sizes.size):
        if count >= target:
            break
        sel[starts[b]:starts[b] + sizes[b]] = 1
        count += int(sizes[b])
    return sel


def reorder_problem(n: int, seed: int = 0, *, select_frac: float = 0.3,
                    q: str = "identity", reflectors: int = 64,
                    clusters: bool = False, spread: float = 1e-6, kappa: float = 1.0,
                    order: str = "F"):
    """One reordering instance: (S, Q, select), S and Q float64, column-major
    (order "F", the default) or row-major (order "C": the same values)."""
    rng = np.random.default_rng(seed)
    S, sizes = schur_form(n, rng, clusters=clusters, spread=spread, kappa=kappa, order=order)
    if q == "identity":
        Q = np.asfortranarray(np.eye(n)) if order == "F" else np.eye(n)
    elif q == "householder":
        Q = householder_q(n, rng, reflectors, order=order)
    else:
        raise ValueError(f"unknown Q kind {q!r}")
    sel = selection(sizes, select_frac, rng)
    return S, Q, sel


# The five workloads (sizes and laws as stated in the module docstring).
def config(name: str, seed: int = 0):
    """Named workloads: 'n400', 'n4000', 'n16000c' (clustered)."""
    if name == "n400":
        return reorder_problem(400, seed, select_frac=0.30, q="identity")
    if name == "n4000":
        return reorder_problem(4000, seed, select_frac=0.35, q="householder")
    if name == "n16000c":
        return reorder_problem(16000, seed, select_frac=0.50, q="householder",
                               clusters=True, spread=1e-6)
    raise ValueError(name)


def batch_problems(count: int, seed: int = 0, nmin: int = 32, nmax: int = 512,
                   pmin: float = 0.2, pmax: float = 0.6):
    """Independent small instances: n ~ U{nmin..nmax}, p ~ U(pmin, pmax),
    Q = product of min(n, 64) reflectors."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, count)
    ps = rng.uniform(pmin, pmax, count)
    seeds = rng.integers(0, 2**62, count)
    return [(int(ns[i]), float(ps[i]), int(seeds[i])) for i in range(count)]


def request_stream(count: int, seed: int = 0, nmin: int = 64, nmax: int = 8192,
                   pmin: float = 0.1, pmax: float = 0.6, rate: float = 1.0):
    """Poisson arrivals (rate per second) of requests with n log-uniform in
    [nmin, nmax] and select fraction U(pmin, pmax)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps)
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), count)).astype(np.int64)
    ps = rng.uniform(pmin, pmax, count)
    seeds = rng.integers(0, 2**62, count)
    return [(float(t[i]), int(ns[i]), float(ps[i]), int(seeds[i])) for i in range(count)]


def serve_base(nmax: int = 8192, seed: int = 0):
    """Base form of the serving requests: (S, sizes, block starts)."""
    rng = np.random.default_rng(seed)
    S, sizes = schur_form(nmax, rng)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return S, sizes, starts


def serve_request(base, n: int, frac: float, seed: int, reflectors: int = 8):
    """One serving request of order about n (the block boundary at or after
    k + n ends it, capped by the base): (S, Q, select), Fortran order."""
    S0, sizes, starts = base
    N = S0.shape[0]
    rng = np.random.default_rng(seed)
    n = int(min(max(n, 1), N))
    last = int(np.searchsorted(starts, N - n, side="right")) - 1
    b0 = int(rng.integers(0, max(last, 0) + 1))
    k = int(starts[b0])
    b1 = int(np.searchsorted(starts, k + n, side="left"))
    e = int(starts[b1]) if b1 < starts.size else N
    S = np.asfortranarray(S0[k:e, k:e])
    Q = householder_q(e - k, rng, reflectors)
    sel = selection(sizes[b0:b1], frac, rng)
    return S, Q, sel


def serve_problem(n: int, frac: float, seed: int, reflectors: int = 8, order: str = "F"):
    """One serving request: an independent form of order n from the seeded
    generator (as reorder_problem), Q of `reflectors` reflectors."""
    return reorder_problem(int(n), seed, select_frac=frac, q="householder",
                           reflectors=reflectors, order=order)


def gen_schur_pair(n: int, rng: np.random.Generator, *, frac_1x1: float = 0.6,
                   clusters: bool = False, spread: float = 1e-6, kappa: float = 1.0):
    """Random generalized real Schur form (S, T). Returns (S, T, sizes).

    clusters / spread / kappa as for schur_form: eigenvalues drawn from 12
    real and 8 complex centres, the standardized 2x2 parts M made non-normal
    by kappa (the combination that produces rejected swaps)."""
    sizes = block_sizes(n, rng, frac_1x1)
    S = np.zeros((n, n), dtype=np.float64, order="F")
    T = np.zeros((n, n), dtype=np.float64, order="F")
    if n == 0:
        return S, T, sizes
    S[:] = np.triu(rng.standard_normal((n, n)), k=1)
    T[:] = np.triu(rng.standard_normal((n, n)), k=1)
    T[np.diag_indices(n)] = rng.uniform(0.5, 2.0, n)
    nb1 = int(np.sum(sizes == 1))
    nb2 = int(np.sum(sizes == 2))
    if clusters:
        rc = rng.standard_normal(12)
        ca = rng.standard_normal(8)
        cb = rng.uniform(0.1, 2.0, 8) * rng.choice([-1.0, 1.0], 8)
        cc = -np.sign(cb) * rng.uniform(0.1, 2.0, 8)
        lam = rc[rng.integers(0, 12, nb1)] + spread * rng.standard_normal(nb1)
        pick = rng.integers(0, 8, nb2)
        a = ca[pick] + spread * rng.standard_normal(nb2)
        b = cb[pick] * (1.0 + spread * rng.standard_normal(nb2))
        c = cc[pick] * (1.0 + spread * rng.standard_normal(nb2))
    else:
        lam = rng.standard_normal(nb1)
        a = rng.standard_normal(nb2)
        b = rng.uniform(0.1, 2.0, nb2) * rng.choice([-1.0, 1.0], nb2)
        c = -np.sign(b) * rng.uniform(0.1, 2.0, nb2)
    if kappa != 1.0:
        b = b * kappa
        c = c / kappa
    i1 = i2 = 0
    pos = 0
    for sz in sizes:
        if sz == 1:
            S[pos, pos] = lam[i1] * T[pos, pos]
            i1 += 1
        else:
            Tb = T[pos:pos + 2, pos:pos + 2]
            M = np.array([[a[i2], b[i2]], [c[i2], a[i2]]])
            S[pos:pos + 2, pos:pos + 2] = Tb @ M
            i2 += 1
        pos += int(sz)
    return S, T, sizes


def gen_problem(n: int, seed: int = 0, *, select_frac: float = 0.3, qz: str = "householder",
                reflectors: int = 64, clusters: bool = False, spread: float = 1e-6,
                kappa: float = 1.0):
    """One generalized reordering instance: (S, T, Q, Z, select)."""
    rng = np.random.default_rng(seed)
    S, T, sizes = gen_schur_pair(n, rng, clusters=clusters, spread=spread, kappa=kappa)
    if qz == "identity":
        Q = np.asfortranarray(np.eye(n))
        Z = np.asfortranarray(np.eye(n))
    elif qz == "householder":
        Q = householder_q(n, rng, reflectors)
        Z = householder_q(n, rng, reflectors)
    else:
        raise ValueError(f"unknown Q/Z kind {qz!r}")
    sel = selection(sizes, select_frac, rng)
    return S, T, Q, Z, sel


def gen_config(name: str, seed: int = 0):
    """Named generalized workloads: 'g400', 'g4000'."""
    if name == "g400":
        return gen_problem(400, seed, select_frac=0.30, qz="householder", reflectors=16)
    if name == "g4000":
        return gen_problem(4000, seed, select_frac=0.35, qz="householder")
    raise ValueError(name)


def hessenberg_problem(n: int, seed: int = 0, *, nshifts: int = 8, reflectors: int = 64,
                       q: str = "householder"):
    """One sweep instance: (H, Q, shifts); shifts complex, nshifts even."""
    rng = np.random.default_rng(seed)
    H = np.asfortranarray(np.triu(rng.standard_normal((n, n)), k=-1))
    if q == "identity":
        Q = np.asfortranarray(np.eye(n))
    else:
        Q = householder_q(n, rng, reflectors)
    sh = []
    for b in range(nshifts // 2):
        if b % 2 == 0:
            a, im = rng.standard_normal(), rng.uniform(0.1, 1.0)
            sh += [complex(a, im), complex(a, -im)]
        else:
            sh += [complex(rng.standard_normal(), 0.0), complex(rng.standard_normal(), 0.0)]
    return H, Q, np.array(sh, dtype=complex)


def sweep_config(name: str, seed: int = 0):
    """Named sweep workloads: 'h4000' (n = 4000, 64 shifts), 'h400'."""
    if name == "h4000":
        return hessenberg_problem(4000, seed, nshifts=64, reflectors=64)
    if name == "h400":
        return hessenberg_problem(400, seed, nshifts=16, reflectors=16)
    raise ValueError(name)
