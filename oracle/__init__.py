"""CPU oracle for real Schur-form eigenvalue reordering -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The GPU library never does; the two
share no code.

The arithmetic lives in `reorder_oracle.c` (plain C, binary64,
-ffp-contract=off): the scalar-update reordering of Section 3.2 / Fig. 1a,
producing the reordered Schur form of Eq. 7; and in `eigvec_oracle.c`: the
eigenvectors of a real Schur form (Eq. 5) by back substitution with
overflow protection; in `gen_oracle.c`: the reordering of a generalized
real Schur form (S, T) with Q and Z (Eq. 7, second form); and in
`sweep_oracle.c`: one bulge-chasing sweep of the Schur reduction (Section
3.2).  This module only compiles them with gcc, marshals
numpy arrays through ctypes, and back-transforms the eigenvectors with one
matrix product (Eq. 6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reorder_oracle.c")
_SRC_EV = os.path.join(_HERE, "eigvec_oracle.c")
_SRC_GEN = os.path.join(_HERE, "gen_oracle.c")
_SRC_SWEEP = os.path.join(_HERE, "sweep_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
# the same sources built with -fopenmp: the long row/column/Q loops of the
# reordering split over the host cores (the CPU baseline's multi-core leg)
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False, src: str = _SRC, out: str = _SO, extra=()) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off)."""
    srcs = [src] + ([_SRC_EV, _SRC_GEN, _SRC_SWEEP] if src == _SRC else [])
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(x)
                                                 for x in srcs):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
           "-o", out + ".tmp", *srcs, "-lm", *extra]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; returns the ctypes CDLL."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    so = path or build()
    lib = ctypes.CDLL(so)
    lib.orc_validate.argtypes = [ctypes.c_int, _dp, ctypes.c_int]
    lib.orc_validate.restype = ctypes.c_int
    lib.orc_eigenvalues.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
    lib.orc_eigenvalues.restype = None
    lib.orc_sylvester.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                  ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp]
    lib.orc_sylvester.restype = ctypes.c_int
    lib.orc_std2.argtypes = [ctypes.c_double] * 4 + [_dp, _dp, _dp]
    lib.orc_std2.restype = None
    lib.orc_swap.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_swap.restype = ctypes.c_int
    lib.orc_reorder.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _ip,
                                _dp, _dp, _ip, ctypes.c_int, ctypes.c_int, _llp, _llp,
                                ctypes.POINTER(ctypes.c_ubyte)]
    lib.orc_reorder.restype = ctypes.c_int
    if hasattr(lib, "orc_eigvec"):
        lib.orc_eigvec.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, ctypes.c_int, _ip]
        lib.orc_eigvec.restype = ctypes.c_int
    if hasattr(lib, "orc_gen_reorder"):
        lib.orc_gen_validate.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int]
        lib.orc_gen_validate.restype = ctypes.c_int
        lib.orc_gen_eigenvalues.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                            _dp, _dp]
        lib.orc_gen_eigenvalues.restype = None
        lib.orc_gen_sylvester.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_gen_sylvester.restype = ctypes.c_double
        lib.orc_gen_swap_local.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                           _dp, _dp, _dp, _dp]
        lib.orc_gen_swap_local.restype = ctypes.c_int
        lib.orc_gen_reorder.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                        _dp, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, _dp,
                                        _ip, ctypes.c_int, _llp, _llp]
        lib.orc_gen_reorder.restype = ctypes.c_int
    if hasattr(lib, "orc_qr_sweep"):
        lib.orc_qr_sweep.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                     ctypes.c_int, _dp, _dp]
        lib.orc_qr_sweep.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def build_omp(force: bool = False) -> str:
    """The oracle built with -fopenmp (same sources, same arithmetic)."""
    return build(force, out=_SO_OMP, extra=("-fopenmp",))


def load_omp():
    """The OpenMP build of the oracle (ctypes CDLL with the same functions);
    pass it as `lib=` to the functions below.  Threads: OMP_NUM_THREADS, else
    all cores the process may run on."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = load(build_omp())
    return _lib_omp


def _f64(a):
    return np.asfortranarray(np.array(a, dtype=np.float64, copy=True))


def _ptr(a):
    return a.ctypes.data_as(_dp)


def validate(S, lib=None) -> int:
    S = _f64(S)
    n = S.shape[0]
    return (lib or load()).orc_validate(n, _ptr(S), max(n, 1))


def eigenvalues(S, lib=None):
    S = _f64(S)
    n = S.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    (lib or load()).orc_eigenvalues(n, _ptr(S), max(n, 1), _ptr(wr), _ptr(wi))
    return wr, wi


def sylvester(T11, T22, T12, lib=None):
    """Solve T11 X - X T22 = gamma T12 (p, q in {1, 2}); returns (X, gamma)."""
    T11, T22, T12 = _f64(np.atleast_2d(T11)), _f64(np.atleast_2d(T22)), _f64(np.atleast_2d(T12))
    p, q = T11.shape[0], T22.shape[0]
    X = np.zeros((2, 2), order="F")
    g = ctypes.c_double(0.0)
    (lib or load()).orc_sylvester(p, q, _ptr(T11), p, _ptr(T22), q, _ptr(T12), p,
                                  _ptr(X), 2, ctypes.byref(g))
    return X[:p, :q].copy(), g.value


def std2(M, lib=None):
    """Standardize a 2x2 block: returns (c, s, N) with N = Z^T M Z,
    Z = [[c, -s], [s, c]]."""
    M = np.asarray(M, dtype=np.float64)
    c = ctypes.c_double()
    s = ctypes.c_double()
    out = np.zeros(4)
    (lib or load()).orc_std2(M[0, 0], M[0, 1], M[1, 0], M[1, 1],
                             ctypes.byref(c), ctypes.byref(s), _ptr(out))
    return c.value, s.value, out.reshape(2, 2, order="F")


def swap(S, j, p, q, Q=None, strong=True, lib=None):
    """Swap the p x p block at j with the q x q block below it.
    Returns (status, S_new, Q_new); status 0 = applied, 1 = rejected."""
    S = _f64(S)
    n = S.shape[0]
    Qp = None
    if Q is not None:
        Q = _f64(Q)
        Qp = _ptr(Q)
    st = (lib or load()).orc_swap(n, _ptr(S), n, Qp, n, j, p, q, 1 if strong else 0)
    return st, S, Q


def reorder(S, Q, select, *, abort=False, strong=True, lib=None):
    """Reorder the Schur form (S, Q) so that the selected eigenvalues lead.

    Returns a dict with S, Q (new arrays), wr, wi, m, status, nswaps, nrej,
    sel (final per-position selection flags)."""
    S = _f64(S)
    n = S.shape[0]
    Qp = None
    if Q is not None:
        Q = _f64(Q)
        Qp = _ptr(Q)
    sel_in = np.ascontiguousarray(np.asarray(select, dtype=np.int32))
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    ns = ctypes.c_longlong(0)
    nr = ctypes.c_longlong(0)
    selout = np.zeros(max(n, 1), dtype=np.uint8)
    st = (lib or load()).orc_reorder(n, _ptr(S), max(n, 1), Qp, max(n, 1),
                                     sel_in.ctypes.data_as(_ip), _ptr(wr), _ptr(wi),
                                     ctypes.byref(m), 1 if abort else 0, 1 if strong else 0,
                                     ctypes.byref(ns), ctypes.byref(nr),
                                     selout.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return dict(S=S, Q=Q, wr=wr, wi=wi, m=m.value, status=st, nswaps=ns.value,
                nrej=nr.value, sel=selout[:n].astype(bool))


def eig_columns(S, select=None):
    """Column kinds of the eigenvector matrix for a selection: 0 = real
    eigenvector, 1 / 2 = real / imaginary part of a complex one (diagonal
    order); with the eigenvalue of each column."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    kinds, lams = [], []
    j = 0
    while j < n:
        nb = 2 if (j + 1 < n and S[j + 1, j] != 0.0) else 1
        sel = True if select is None else (select[j] != 0 or (nb == 2 and select[j + 1] != 0))
        if sel:
            if nb == 1:
                kinds.append(0)
                lams.append(complex(S[j, j]))
            else:
                w = np.sqrt(-S[j, j + 1] * S[j + 1, j])
                kinds += [1, 2]
                lams += [complex(S[j, j], w)] * 2
        j += nb
    return np.array(kinds, dtype=np.int32), np.array(lams)


def normalize_columns(X, kinds):
    """max |x_i| = 1 per real column; max(|re| + |im|) = 1 per complex pair."""
    X = np.array(X, dtype=np.float64, copy=True)
    c = 0
    while c < X.shape[1]:
        if kinds[c] == 0:
            m = np.max(np.abs(X[:, c]))
            if m > 0:
                X[:, c] /= m
            c += 1
        else:
            m = np.max(np.abs(X[:, c]) + np.abs(X[:, c + 1]))
            if m > 0:
                X[:, c:c + 2] /= m
            c += 2
    return X


def eigenvectors(S, Q=None, select=None, lib=None):
    """Eigenvectors (Eq. 5) of the real Schur form S for the selected
    eigenvalues, back-transformed by Q (Eq. 6) if given, then normalized.
    Returns (X n x m, column kinds, eigenvalue per column, scalings per column)."""
    S = _f64(S)
    n = S.shape[0]
    kinds, lams = eig_columns(S, select)
    m = len(kinds)
    Y = np.zeros((n, max(m, 1)), dtype=np.float64, order="F")
    ns = np.zeros(max(m, 1), dtype=np.int32)
    sel = None if select is None else np.ascontiguousarray(np.asarray(select, dtype=np.int32))
    got = (lib or load()).orc_eigvec(n, _ptr(S), max(n, 1),
                                     sel.ctypes.data_as(_ip) if sel is not None else None,
                                     _ptr(Y), max(n, 1), ns.ctypes.data_as(_ip))
    assert got == m
    Y = Y[:, :m]
    if Q is not None:
        Y = normalize_columns(np.asarray(Q, dtype=np.float64) @ Y, kinds)
    return Y, kinds, lams, ns[:m]


# ---------------------------------------------------------------------------
# Generalized real Schur form (S, T)
# ---------------------------------------------------------------------------
def gen_validate(S, T, lib=None) -> int:
    S, T = _f64(S), _f64(T)
    n = S.shape[0]
    return (lib or load()).orc_gen_validate(n, _ptr(S), max(n, 1), _ptr(T), max(n, 1))


def gen_eigenvalues(S, T, lib=None):
    """Generalized eigenvalues of the diagonal blocks, diagonal order."""
    S, T = _f64(S), _f64(T)
    n = S.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    (lib or load()).orc_gen_eigenvalues(n, _ptr(S), max(n, 1), _ptr(T), max(n, 1), _ptr(wr),
                                        _ptr(wi))
    return wr + 1j * wi


def gen_sylvester(A, B, p, q, lib=None):
    """Solve A11 R - L A22 = -gamma A12, B11 R - L B22 = -gamma B12 for the
    (p + q) x (p + q) pair (A, B); returns (R, L, gamma)."""
    k = p + q
    DA = np.zeros((4, 4), order="F")
    DB = np.zeros((4, 4), order="F")
    DA[:k, :k] = A
    DB[:k, :k] = B
    R = np.zeros(4)
    L = np.zeros(4)
    g = (lib or load()).orc_gen_sylvester(p, q, _ptr(DA), _ptr(DB), _ptr(R), _ptr(L))
    return (R[:p * q].reshape((p, q), order="F"), L[:p * q].reshape((p, q), order="F"), g)


def gen_swap_local(A, B, p, q, strong=True, lib=None):
    """Swap on a (p + q) x (p + q) pair alone: (status, Qs, Zs, A_new, B_new)."""
    k = p + q
    DA = np.zeros((4, 4), order="F")
    DB = np.zeros((4, 4), order="F")
    DA[:k, :k] = A
    DB[:k, :k] = B
    out = [np.zeros((4, 4), order="F") for _ in range(4)]
    st = (lib or load()).orc_gen_swap_local(p, q, _ptr(DA), _ptr(DB), 1 if strong else 0,
                                            *[_ptr(o) for o in out])
    return (st,) + tuple(o[:k, :k].copy() for o in out)


def gen_reorder(S, T, Q, Z, select, *, strong=True, lib=None):
    """Reorder the generalized Schur form (S, T) with Q, Z so that the
    selected eigenvalues lead.  Returns a dict with S, T, Q, Z (new arrays),
    eigs (complex), m, status, nswaps, nrej."""
    S, T = _f64(S), _f64(T)
    n = S.shape[0]
    Qp = Zp = None
    if Q is not None:
        Q = _f64(Q)
        Qp = _ptr(Q)
    if Z is not None:
        Z = _f64(Z)
        Zp = _ptr(Z)
    sel_in = np.ascontiguousarray(np.asarray(select, dtype=np.int32))
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    ns = ctypes.c_longlong(0)
    nr = ctypes.c_longlong(0)
    ld = max(n, 1)
    st = (lib or load()).orc_gen_reorder(n, _ptr(S), ld, _ptr(T), ld, Qp, ld, Zp, ld,
                                         sel_in.ctypes.data_as(_ip), _ptr(wr), _ptr(wi),
                                         ctypes.byref(m), 1 if strong else 0,
                                         ctypes.byref(ns), ctypes.byref(nr))
    return dict(S=S, T=T, Q=Q, Z=Z, eigs=wr + 1j * wi, m=m.value, status=st,
                nswaps=ns.value, nrej=nr.value)


# ---------------------------------------------------------------------------
# Bulge-chasing sweep on an upper Hessenberg matrix
# ---------------------------------------------------------------------------
def qr_sweep(H, Q, shifts, lib=None):
    """One pipelined multishift sweep on H (upper Hessenberg) with the given
    complex shifts (pairs: real or conjugate).  Returns (status, H_new,
    Q_new)."""
    H = _f64(H)
    n = H.shape[0]
    Qp = None
    if Q is not None:
        Q = _f64(Q)
        Qp = _ptr(Q)
    sh = np.asarray(shifts, dtype=complex).reshape(-1)
    sr = np.ascontiguousarray(sh.real, dtype=np.float64)
    si = np.ascontiguousarray(sh.imag, dtype=np.float64)
    st = (lib or load()).orc_qr_sweep(n, _ptr(H), max(n, 1), Qp, max(n, 1), int(sh.size),
                                      _ptr(sr), _ptr(si))
    return st, H, Q
