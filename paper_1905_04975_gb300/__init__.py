"""gbreorder: eigenvalue reordering of a real Schur form on one GB300 GPU.

Thin ctypes binding over the C ABI declared in include/gbreorder.h
(libgbreorder.so, built in-tree by `build.py`).  It only marshals arguments:
every step of the reordering runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams only.

Matrices are FP64 and column-major.  On the device they are torch tensors
whose memory is column-major: shape (n, n) with strides (1, ld), e.g.
`torch.from_numpy(S_fortran).cuda()` or `to_device(S)` below.  There is no
CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libgbreorder.so")

PREC_DMMA = 0
PREC_OZAKI = 1
PREC_FMA = 2
_PREC = {"dmma": PREC_DMMA, "ozaki": PREC_OZAKI, "fma": PREC_FMA}
ON_REJECT_CONTINUE = 0
ON_REJECT_ABORT = 1
SCHED_PERSISTENT = 0
SCHED_SEQUENTIAL = 1
INJECT_STALL = 1

ERR_CUDA = -1001
ERR_NOMEM = -1002
ERR_TIMEOUT = -1003
ERR_UNSUPPORTED = -1004
ERR_NOALLOC_LIMIT = -1005
ERR_PLAN_MISMATCH = -1006
ERR_CAPTURING = -1007
NOALLOC_MAX_N = 16384
AUTO = 0


class GbrOpts(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("chain", ctypes.c_int), ("precision", ctypes.c_int),
                ("slices", ctypes.c_int), ("strong_test", ctypes.c_int),
                ("on_reject", ctypes.c_int), ("validate", ctypes.c_int),
                ("timing", ctypes.c_int), ("sched", ctypes.c_int), ("inject", ctypes.c_int),
                ("wait_limit_ms", ctypes.c_longlong)]


class GbrStats(ctypes.Structure):
    _fields_ = [("swaps", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("windows", ctypes.c_longlong), ("chains", ctypes.c_longlong),
                ("launches", ctypes.c_longlong), ("upd_flops", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_window", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_sched", ctypes.c_double),
                ("win_flops", ctypes.c_double), ("tasks", ctypes.c_longlong),
                ("sched_cp_ms", ctypes.c_double), ("sched_sim_ms", ctypes.c_double),
                ("ms_graph", ctypes.c_double), ("ms_order", ctypes.c_double),
                ("upd_flops_issued", ctypes.c_double), ("ms_h2d", ctypes.c_double),
                ("ms_d2h", ctypes.c_double)]


class GbrServerCfg(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_longlong), ("max_inflight", ctypes.c_int),
                ("sms", ctypes.c_int), ("ring_entries", ctypes.c_longlong),
                ("idle_limit_ms", ctypes.c_longlong), ("device", ctypes.c_int),
                ("opts", GbrOpts)]


class GbrServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("passes", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("req_per_s", ctypes.c_double), ("eigs_per_s", ctypes.c_double),
                ("mean_inflight", ctypes.c_double), ("peak_mem_bytes", ctypes.c_double)]


# Every symbol the header declares, with (restype, argtypes).
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_REORDER_ARGS = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _ip,
                 _dp, _dp, _ip, ctypes.POINTER(GbrOpts), ctypes.POINTER(GbrStats),
                 ctypes.c_void_p]
_REORDER_GEN_ARGS = [ctypes.c_int] + [ctypes.c_void_p, ctypes.c_int] * 4 + [
    _ip, _dp, _dp, _ip, ctypes.POINTER(GbrOpts), ctypes.POINTER(GbrStats), ctypes.c_void_p]
SYMBOLS = {
    "gbr_default_opts": (None, [ctypes.POINTER(GbrOpts)]),
    "gbr_reorder_gen": (ctypes.c_int, _REORDER_GEN_ARGS),
    "gbr_plan_sweep": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip,
                                      ctypes.c_int]),
    "gbr_qr_sweep": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_int, _dp, _dp,
                                    ctypes.POINTER(GbrOpts), ctypes.POINTER(GbrStats),
                                    ctypes.c_void_p]),
    "gbr_reorder_gen_host": (ctypes.c_int, _REORDER_GEN_ARGS),
    "gbr_reorder": (ctypes.c_int, _REORDER_ARGS),
    "gbr_reorder_host": (ctypes.c_int, _REORDER_ARGS),
    "gbr_reorder_noalloc": (ctypes.c_int, _REORDER_ARGS),
    "gbr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gbr_last_error": (ctypes.c_char_p, []),
    "gbr_release": (None, []),
    "gbr_pool_bytes": (ctypes.c_longlong, []),
    "gbr_version": (ctypes.c_int, []),
    "gbr_last_trace": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "gbr_eigenvectors": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_void_p,
                                        ctypes.c_int, _ip, _ip, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "gbr_update_panel": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "gbr_plan": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte), _ip, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, _ip, _dp]),
    "gbr_batch_create": (ctypes.c_int, [ctypes.c_int, _ip, ctypes.POINTER(ctypes.c_void_p), _ip,
                                        ctypes.POINTER(ctypes.c_void_p), _ip, _ip,
                                        ctypes.POINTER(GbrOpts), _ip,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "gbr_batch_run": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _ip, _ip,
                                     ctypes.POINTER(GbrStats), ctypes.c_void_p]),
    "gbr_batch_destroy": (None, [ctypes.c_void_p]),
    "gbr_reorder_batched": (ctypes.c_int, [ctypes.c_int, _ip, ctypes.POINTER(ctypes.c_void_p), _ip,
                                           ctypes.POINTER(ctypes.c_void_p), _ip, _ip, _dp, _dp,
                                           _ip, _ip, ctypes.POINTER(GbrOpts),
                                           ctypes.POINTER(GbrStats), ctypes.c_void_p]),
    "gbr_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "gbr_tune_get": (ctypes.c_int, [ctypes.c_int, _ip, _ip, _ip]),
    "gbr_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "gbr_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "gbr_server_default_cfg": (None, [ctypes.POINTER(GbrServerCfg)]),
    "gbr_server_create": (ctypes.c_int, [ctypes.POINTER(GbrServerCfg),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "gbr_server_submit": (ctypes.c_longlong, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                              ctypes.c_int, _ip, _dp, _dp]),
    "gbr_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, _ip, _ip]),
    "gbr_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, _ip, _ip,
                                       ctypes.c_longlong]),
    "gbr_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(GbrServerStats)]),
    "gbr_server_destroy": (None, [ctypes.c_void_p]),
}

_lib = None


def load(path: str = SO_PATH):
    """Load libgbreorder.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path == SO_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m "
                          "paper_1905_04975_gb300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == SO_PATH:
        _lib = lib
    return lib


class GbrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gbr status {status}: {msg}")
        self.status = status


def status_string(status: int) -> str:
    lib = load()
    s = lib.gbr_status_string(status).decode()
    if status in (ERR_CUDA, ERR_NOMEM):
        s += f" ({lib.gbr_last_error().decode()})"
    return s


def default_opts() -> GbrOpts:
    o = GbrOpts()
    load().gbr_default_opts(ctypes.byref(o))
    return o


def make_opts(window=None, chain=None, precision=None, slices=None, strong=None,
              validate=None, timing=None, sched=None, inject=None, wait_limit_ms=None,
              on_reject=None) -> GbrOpts:
    o = default_opts()
    if on_reject is not None:
        o.on_reject = {"continue": ON_REJECT_CONTINUE, "abort": ON_REJECT_ABORT}.get(on_reject,
                                                                                     on_reject)
    if window is not None:
        o.window = int(window)
    if chain is not None:
        o.chain = int(chain)
    if precision is not None:
        o.precision = _PREC.get(precision, precision)
    if slices is not None:
        o.slices = int(slices)
    if strong is not None:
        o.strong_test = 1 if strong else 0
    if validate is not None:
        o.validate = 1 if validate else 0
    if timing is not None:
        o.timing = int(timing) if not isinstance(timing, bool) else int(timing)
    if sched is not None:
        o.sched = {"persistent": SCHED_PERSISTENT, "sequential": SCHED_SEQUENTIAL}.get(sched, sched)
    if inject is not None:
        o.inject = int(inject)
    if wait_limit_ms is not None:
        o.wait_limit_ms = int(wait_limit_ms)
    return o


@dataclass
class ReorderResult:
    status: int           # 0, or number of rejected swaps (> 0)
    m: int                # number of selected eigenvalues
    eigs: np.ndarray      # complex eigenvalues of the result, diagonal order
    stats: GbrStats


def _colmajor_ld(t) -> int:
    n0, n1 = t.shape
    if str(t.dtype) != "torch.float64":
        raise TypeError("matrices must be float64")
    if n0 > 1 and t.stride(0) != 1:
        raise ValueError("matrix must be column-major (stride (1, ld)); use to_device()")
    return max(t.stride(1), max(n0, 1)) if n1 > 1 else max(n0, 1)


def to_device(A: np.ndarray, device="cuda"):
    """Copy a numpy matrix to a column-major CUDA float64 tensor."""
    import torch
    A = np.asfortranarray(A, dtype=np.float64)
    t = torch.empty((A.shape[1], A.shape[0]), dtype=torch.float64, device=device).t()
    t.copy_(torch.from_numpy(A))
    return t


def to_host(t) -> np.ndarray:
    """Copy a column-major CUDA tensor back to a Fortran-ordered numpy array."""
    return np.asfortranarray(t.cpu().numpy())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def _finish(rc, n, m, wr, wi, stats, allow_partial):
    if rc < 0 or (rc > 0 and not allow_partial):
        raise GbrError(rc, status_string(rc))
    return ReorderResult(status=rc, m=m.value, eigs=wr + 1j * wi, stats=stats)


def reorder(S, Q, select, *, opts: GbrOpts | None = None, stream=None, allow_partial=True,
            **kw) -> ReorderResult:
    """Reorder (S, Q) in place on the GPU so that the selected eigenvalues lead.

    S, Q: column-major float64 CUDA tensors (Q may be None); select: ints,
    one per diagonal position.  Keyword options: window, chain, precision,
    strong, validate."""
    lib = load()
    n = int(S.shape[0])
    ldS = _colmajor_ld(S)
    qptr, ldQ = None, max(n, 1)
    if Q is not None:
        ldQ = _colmajor_ld(Q)
        qptr = ctypes.c_void_p(Q.data_ptr())
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    if sel.size != n:
        raise ValueError("select must have n entries")
    o = opts if opts is not None else make_opts(**kw)
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    stats = GbrStats()
    rc = lib.gbr_reorder(n, ctypes.c_void_p(S.data_ptr()), ldS, qptr, ldQ,
                         sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                         wi.ctypes.data_as(_dp), ctypes.byref(m), ctypes.byref(o),
                         ctypes.byref(stats), _stream_handle(stream))
    return _finish(rc, n, m, wr, wi, stats, allow_partial)


def update_panel(Y, U, precision="dmma", *, stream=None) -> None:
    """Y <- Y U in place on the GPU (one off-diagonal update of a window).

    Y: 2-D float64 CUDA tensor (rows x w) with stride 1 along one dimension
    (row- or column-major); U: w x w column-major float64 CUDA tensor.
    precision: "dmma" (FP64 tensor cores) or "ozaki" (emulated FP64 on the
    bf16 tensor cores)."""
    lib = load()
    rows, w = int(Y.shape[0]), int(Y.shape[1])
    if str(Y.dtype) != "torch.float64" or str(U.dtype) != "torch.float64":
        raise TypeError("Y and U must be float64")
    if tuple(U.shape) != (w, w):
        raise ValueError("U must be w x w")
    ldU = _colmajor_ld(U)
    prec = _PREC.get(precision, precision)
    rc = lib.gbr_update_panel(rows, w, ctypes.c_void_p(Y.data_ptr()), int(Y.stride(0)),
                              int(Y.stride(1)), ctypes.c_void_p(U.data_ptr()), ldU, int(prec),
                              _stream_handle(stream))
    if rc != 0:
        raise GbrError(rc, status_string(rc))


class GbrEvStats(ctypes.Structure):
    _fields_ = [("ms_solve", ctypes.c_double), ("ms_backtransform", ctypes.c_double),
                ("ms_normalize", ctypes.c_double), ("solve_flops", ctypes.c_double),
                ("backtransform_flops", ctypes.c_double)]


def eigenvectors(S, Q=None, select=None, *, stream=None, with_scalings=False, stats=None,
                 out=None):
    """Eigenvectors of the real Schur form S (column-major float64 CUDA
    tensor) for the selected eigenvalues (None: all), back-transformed by Q
    if given, normalized; returns an n x m column-major CUDA tensor (a
    conjugate pair gives its real and imaginary part as two columns), and
    with with_scalings also the per-column count of 2^-512 scalings.  stats:
    a GbrEvStats to fill with kernel times and algorithmic flops."""
    import torch
    lib = load()
    n = int(S.shape[0])
    ldS = _colmajor_ld(S)
    qptr, ldQ = None, max(n, 1)
    if Q is not None:
        ldQ = _colmajor_ld(Q)
        qptr = ctypes.c_void_p(Q.data_ptr())
    sel = None
    if select is not None:
        sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
        if sel.size != n:
            raise ValueError("select must have n entries")
    selp = sel.ctypes.data_as(_ip) if sel is not None else None
    m = ctypes.c_int(0)
    st = _stream_handle(stream)
    if out is None:
        rc = lib.gbr_eigenvectors(n, ctypes.c_void_p(S.data_ptr()), ldS, qptr, ldQ, selp, None,
                                  max(n, 1), ctypes.byref(m), None, None, st)
        if rc != 0:
            raise GbrError(rc, status_string(rc))
        X = torch.zeros((max(m.value, 1), max(n, 1)), dtype=torch.float64, device=S.device).t()
        X = X[:n, : m.value]
    else:
        X = out
        m.value = int(out.shape[1])
    ns = np.zeros(max(m.value, 1), dtype=np.int32)
    if m.value > 0:
        rc = lib.gbr_eigenvectors(n, ctypes.c_void_p(S.data_ptr()), ldS, qptr, ldQ, selp,
                                  ctypes.c_void_p(X.data_ptr()), _colmajor_ld(X), ctypes.byref(m),
                                  ns.ctypes.data_as(_ip),
                                  ctypes.byref(stats) if stats is not None else None, st)
        if rc != 0:
            raise GbrError(rc, status_string(rc))
    return (X, ns[: m.value]) if with_scalings else X


def reorder_noalloc(S, Q, select, *, opts: GbrOpts | None = None, stream=None,
                    allow_partial=True, **kw) -> ReorderResult:
    """Same as reorder(), through gbr_reorder_noalloc: no device allocation;
    scratch comes from a fixed array in the library image (n <= 16384)."""
    lib = load()
    n = int(S.shape[0])
    ldS = _colmajor_ld(S)
    qptr, ldQ = None, max(n, 1)
    if Q is not None:
        ldQ = _colmajor_ld(Q)
        qptr = ctypes.c_void_p(Q.data_ptr())
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    o = opts if opts is not None else make_opts(**kw)
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    stats = GbrStats()
    rc = lib.gbr_reorder_noalloc(n, ctypes.c_void_p(S.data_ptr()), ldS, qptr, ldQ,
                                 sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                                 wi.ctypes.data_as(_dp), ctypes.byref(m), ctypes.byref(o),
                                 ctypes.byref(stats), _stream_handle(stream))
    return _finish(rc, n, m, wr, wi, stats, allow_partial)


def reorder_host(S: np.ndarray, Q: np.ndarray | None, select, *, opts: GbrOpts | None = None,
                 stream=None, allow_partial=True, **kw) -> ReorderResult:
    """Same as reorder() for host (numpy, Fortran-ordered float64) S and Q,
    updated in place; the library copies them to the GPU and back."""
    lib = load()
    if not (S.flags.f_contiguous and S.dtype == np.float64):
        raise ValueError("S must be a Fortran-ordered float64 array")
    n = int(S.shape[0])
    qptr = None
    if Q is not None:
        if not (Q.flags.f_contiguous and Q.dtype == np.float64):
            raise ValueError("Q must be a Fortran-ordered float64 array")
        qptr = ctypes.c_void_p(Q.ctypes.data)
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    o = opts if opts is not None else make_opts(**kw)
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    stats = GbrStats()
    rc = lib.gbr_reorder_host(n, ctypes.c_void_p(S.ctypes.data), max(n, 1), qptr, max(n, 1),
                              sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                              wi.ctypes.data_as(_dp), ctypes.byref(m), ctypes.byref(o),
                              ctypes.byref(stats), _stream_handle(stream))
    return _finish(rc, n, m, wr, wi, stats, allow_partial)


def _gen_opts(opts, kw):
    return opts if opts is not None else make_opts(**kw)


def reorder_gen(S, T, Q, Z, select, *, opts: GbrOpts | None = None, stream=None,
                allow_partial=True, **kw) -> ReorderResult:
    """Reorder the generalized Schur form (S, T) in place on the GPU so that
    the selected generalized eigenvalues lead; Q <- Q Q3, Z <- Z Z3.

    S, T, Q, Z: column-major float64 CUDA tensors (Q, Z may be None).
    Keyword options as for reorder(); window is capped at 64."""
    lib = load()
    n = int(S.shape[0])
    ptrs = []
    for X in (S, T, Q, Z):
        if X is None:
            ptrs += [None, max(n, 1)]
        else:
            ptrs += [ctypes.c_void_p(X.data_ptr()), _colmajor_ld(X)]
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    if sel.size != n:
        raise ValueError("select must have n entries")
    o = _gen_opts(opts, kw)
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    stats = GbrStats()
    rc = lib.gbr_reorder_gen(n, *ptrs, sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                             wi.ctypes.data_as(_dp), ctypes.byref(m), ctypes.byref(o),
                             ctypes.byref(stats), _stream_handle(stream))
    return _finish(rc, n, m, wr, wi, stats, allow_partial)


def reorder_gen_host(S, T, Q, Z, select, *, opts: GbrOpts | None = None, stream=None,
                     allow_partial=True, **kw) -> ReorderResult:
    """reorder_gen() for host (numpy, Fortran-ordered float64) matrices,
    updated in place; the library copies them to the GPU and back."""
    lib = load()
    n = int(S.shape[0])
    ptrs = []
    for X in (S, T, Q, Z):
        if X is None:
            ptrs += [None, max(n, 1)]
            continue
        if not (X.flags.f_contiguous and X.dtype == np.float64):
            raise ValueError("matrices must be Fortran-ordered float64 arrays")
        ptrs += [ctypes.c_void_p(X.ctypes.data), max(n, 1)]
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    o = _gen_opts(opts, kw)
    wr = np.zeros(n)
    wi = np.zeros(n)
    m = ctypes.c_int(0)
    stats = GbrStats()
    rc = lib.gbr_reorder_gen_host(n, *ptrs, sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                                  wi.ctypes.data_as(_dp), ctypes.byref(m), ctypes.byref(o),
                                  ctypes.byref(stats), _stream_handle(stream))
    return _finish(rc, n, m, wr, wi, stats, allow_partial)


@dataclass
class SweepResult:
    status: int
    stats: GbrStats


def qr_sweep(H, Q, shifts, *, opts: GbrOpts | None = None, stream=None, **kw) -> SweepResult:
    """One bulge-chasing sweep on the upper Hessenberg H (column-major float64
    CUDA tensor) with the given complex shifts (pairs: two real shifts or a
    conjugate pair); H and Q (or None) are updated in place.  Keyword
    options: window (<= 96, default 64), chain (shifts per chain, default
    16), sched, validate, timing."""
    lib = load()
    n = int(H.shape[0])
    ldH = _colmajor_ld(H)
    qptr, ldQ = None, max(n, 1)
    if Q is not None:
        ldQ = _colmajor_ld(Q)
        qptr = ctypes.c_void_p(Q.data_ptr())
    sh = np.asarray(shifts, dtype=complex).reshape(-1)
    sr = np.ascontiguousarray(sh.real, dtype=np.float64)
    si = np.ascontiguousarray(sh.imag, dtype=np.float64)
    if opts is None:
        kw.setdefault("window", 64)
        kw.setdefault("chain", 16)
    o = opts if opts is not None else make_opts(**kw)
    stats = GbrStats()
    rc = lib.gbr_qr_sweep(n, ctypes.c_void_p(H.data_ptr()), ldH, qptr, ldQ, int(sh.size),
                          sr.ctypes.data_as(_dp), si.ctypes.data_as(_dp), ctypes.byref(o),
                          ctypes.byref(stats), _stream_handle(stream))
    if rc < 0:
        raise GbrError(rc, status_string(rc))
    return SweepResult(status=rc, stats=stats)


def plan_sweep(n, nshifts, window=64, chain=16):
    """Host-only window plan of a bulge-chasing sweep: int array (k x 6) of
    (s, e, t0, t1, b0, nb) per window, in program order."""
    lib = load()
    cnt = lib.gbr_plan_sweep(int(n), int(nshifts), int(window), int(chain), None, 0)
    if cnt < 0:
        raise GbrError(cnt, "invalid sweep plan arguments")
    out = np.zeros(6 * max(cnt, 1), dtype=np.int32)
    cnt = lib.gbr_plan_sweep(int(n), int(nshifts), int(window), int(chain), out.ctypes.data_as(_ip),
                             cnt)
    return out[:6 * cnt].reshape(cnt, 6)


def plan(sub, select, window=128, chain=64, with_q=True):
    """Host-only window plan: returns (windows (k x 2 int array of [s, e)),
    chains, update flops)."""
    lib = load()
    sub = np.ascontiguousarray(np.asarray(sub, dtype=np.uint8).reshape(-1))
    sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
    n = sub.size
    ch = ctypes.c_int(0)
    fl = ctypes.c_double(0.0)
    cnt = lib.gbr_plan(n, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), sel.ctypes.data_as(_ip),
                       window, chain, 1 if with_q else 0, None, 0, None, None)
    if cnt < 0:
        raise GbrError(cnt, "invalid plan arguments")
    out = np.zeros(2 * max(cnt, 1), dtype=np.int32)
    cnt = lib.gbr_plan(n, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), sel.ctypes.data_as(_ip),
                       window, chain, 1 if with_q else 0, out.ctypes.data_as(_ip), cnt,
                       ctypes.byref(ch), ctypes.byref(fl))
    return out[:2 * cnt].reshape(cnt, 2), ch.value, fl.value


def last_trace() -> np.ndarray:
    """Per-task timeline of the last persistent launch made with timing=2:
    int64 array (tasks x 8): kind, window, y0, rows, sm, take_ns, start_ns, end_ns."""
    lib = load()
    nt = lib.gbr_last_trace(None, 0)
    out = np.zeros((max(nt, 0), 8), dtype=np.int64)
    if nt > 0:
        lib.gbr_last_trace(out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), nt)
    return out


# ---------------------------------------------------------------------------
# Batched reordering
# ---------------------------------------------------------------------------
@dataclass
class BatchResult:
    status: np.ndarray    # per instance: 0, +k rejected swaps, -2 invalid
    m: np.ndarray         # selected eigenvalues per instance
    eigs: list            # per instance: complex eigenvalues in diagonal order
    stats: GbrStats
    rc: int               # 0, or the number of instances with rejected swaps


def _batch_args(S_list, Q_list, selects):
    count = len(S_list)
    n = np.array([int(S.shape[0]) for S in S_list], dtype=np.int32)
    ldS = np.array([_colmajor_ld(S) for S in S_list], dtype=np.int32)
    Sp = (ctypes.c_void_p * max(count, 1))(*[S.data_ptr() for S in S_list])
    Qp = None
    ldQ = None
    if Q_list is not None:
        Qp = (ctypes.c_void_p * max(count, 1))(*[(Q.data_ptr() if Q is not None else None)
                                                 for Q in Q_list])
        ldQ = np.array([(_colmajor_ld(Q) if Q is not None else 1) for Q in Q_list], dtype=np.int32)
    sel = [np.asarray(s, dtype=np.int32).reshape(-1) for s in selects]
    for s_, nn in zip(sel, n):
        if s_.size != nn:
            raise ValueError("each selection must have n entries")
    selc = np.ascontiguousarray(np.concatenate(sel) if sel else np.zeros(1, np.int32))
    return count, n, ldS, Sp, Qp, ldQ, selc


class Batch:
    """A planned batch (gbr_batch_create): one task graph over all instances
    and a captured CUDA graph; run() reorders the current contents of the
    tensors in place (same block structure as at planning)."""

    def __init__(self, S_list, Q_list, selects, *, opts: GbrOpts | None = None, stream=None,
                 **kw):
        lib = load()
        self._args = _batch_args(S_list, Q_list, selects)
        count, n, ldS, Sp, Qp, ldQ, selc = self._args
        self._keep = (S_list, Q_list)
        self.n = n
        o = opts if opts is not None else make_opts(**kw)
        self.create_status = np.zeros(max(count, 1), dtype=np.int32)
        h = ctypes.c_void_p(None)
        rc = lib.gbr_batch_create(count, n.ctypes.data_as(_ip), Sp, ldS.ctypes.data_as(_ip), Qp,
                                  ldQ.ctypes.data_as(_ip) if ldQ is not None else None,
                                  selc.ctypes.data_as(_ip), ctypes.byref(o),
                                  self.create_status.ctypes.data_as(_ip), ctypes.byref(h),
                                  _stream_handle(stream))
        if rc != 0:
            raise GbrError(rc, status_string(rc))
        self._h = h

    def run(self, stream=None) -> BatchResult:
        lib = load()
        count = len(self.n)
        tot = int(self.n.sum())
        wr = np.zeros(max(tot, 1))
        wi = np.zeros(max(tot, 1))
        m = np.zeros(max(count, 1), dtype=np.int32)
        st = np.zeros(max(count, 1), dtype=np.int32)
        stats = GbrStats()
        rc = lib.gbr_batch_run(self._h, wr.ctypes.data_as(_dp), wi.ctypes.data_as(_dp),
                               m.ctypes.data_as(_ip), st.ctypes.data_as(_ip), ctypes.byref(stats),
                               _stream_handle(stream))
        if rc < 0:
            raise GbrError(rc, status_string(rc))
        off = np.concatenate([[0], np.cumsum(self.n)])
        eigs = [wr[off[i]:off[i + 1]] + 1j * wi[off[i]:off[i + 1]] for i in range(count)]
        return BatchResult(status=st[:count], m=m[:count], eigs=eigs, stats=stats, rc=rc)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gbr_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reorder_batched(S_list, Q_list, selects, *, opts: GbrOpts | None = None, stream=None,
                    **kw) -> BatchResult:
    """One-shot batched reorder (gbr_reorder_batched) of lists of column-major
    CUDA tensors (Q_list may be None, or hold None entries); window/chain
    AUTO (0) takes the autotuner's choice per instance."""
    lib = load()
    count, n, ldS, Sp, Qp, ldQ, selc = _batch_args(S_list, Q_list, selects)
    o = opts if opts is not None else make_opts(**kw)
    tot = int(n.sum())
    wr = np.zeros(max(tot, 1))
    wi = np.zeros(max(tot, 1))
    m = np.zeros(max(count, 1), dtype=np.int32)
    st = np.zeros(max(count, 1), dtype=np.int32)
    stats = GbrStats()
    rc = lib.gbr_reorder_batched(count, n.ctypes.data_as(_ip), Sp, ldS.ctypes.data_as(_ip), Qp,
                                 ldQ.ctypes.data_as(_ip) if ldQ is not None else None,
                                 selc.ctypes.data_as(_ip), wr.ctypes.data_as(_dp),
                                 wi.ctypes.data_as(_dp), m.ctypes.data_as(_ip),
                                 st.ctypes.data_as(_ip), ctypes.byref(o), ctypes.byref(stats),
                                 _stream_handle(stream))
    if rc < 0:
        raise GbrError(rc, status_string(rc))
    off = np.concatenate([[0], np.cumsum(n)])
    eigs = [wr[off[i]:off[i + 1]] + 1j * wi[off[i]:off[i + 1]] for i in range(count)]
    return BatchResult(status=st[:count], m=m[:count], eigs=eigs, stats=stats, rc=rc)


def autotune(n_max: int, per_class: int = 256, stream=None) -> int:
    """Run the batched-path autotuner for sizes up to n_max on the current
    device; returns the number of size classes tuned."""
    rc = load().gbr_autotune(int(n_max), int(per_class), _stream_handle(stream))
    if rc < 0:
        raise GbrError(rc, status_string(rc))
    return rc


def tune_get(n: int):
    """(window, chain, far tile rows, tuned?) the batched path uses for order n."""
    w, m, t = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    tuned = load().gbr_tune_get(int(n), ctypes.byref(w), ctypes.byref(m), ctypes.byref(t))
    return w.value, m.value, t.value, bool(tuned)


def tune_save(path) -> int:
    """Write the current device's autotuner table to a JSON file (gbr_tune_save);
    returns the number of size classes written."""
    rc = load().gbr_tune_save(os.fsencode(path))
    if rc < 0:
        raise GbrError(rc, "tune_save: cannot write " + str(path))
    return rc


def tune_load(path) -> int:
    """Load a table written by tune_save into the current device's autotuner
    table (gbr_tune_load); returns the number of size classes loaded."""
    rc = load().gbr_tune_load(os.fsencode(path))
    if rc < 0:
        raise GbrError(rc, "tune_load: cannot read or invalid " + str(path))
    return rc


# ---------------------------------------------------------------------------
# Reordering server (continuous batching)
# ---------------------------------------------------------------------------
def server_cfg(mem_cap_bytes=None, max_inflight=None, sms=None, ring_entries=None,
               idle_limit_ms=None, device=None, opts: GbrOpts | None = None,
               **kw) -> GbrServerCfg:
    c = GbrServerCfg()
    load().gbr_server_default_cfg(ctypes.byref(c))
    for name, v in (("mem_cap_bytes", mem_cap_bytes), ("max_inflight", max_inflight),
                    ("sms", sms), ("ring_entries", ring_entries),
                    ("idle_limit_ms", idle_limit_ms), ("device", device)):
        if v is not None:
            setattr(c, name, int(v))
    c.opts = opts if opts is not None else make_opts(**kw)
    return c


class Server:
    """gbr_server: submit host (numpy, Fortran-ordered float64) S and Q;
    they are overwritten in place when the request completes.  The object
    keeps every buffer of a request alive until it has completed."""

    def __init__(self, cfg: GbrServerCfg | None = None, **kw):
        lib = load()
        self._cfg = cfg if cfg is not None else server_cfg(**kw)
        h = ctypes.c_void_p(None)
        rc = lib.gbr_server_create(ctypes.byref(self._cfg), ctypes.byref(h))
        if rc != 0:
            raise GbrError(rc, status_string(rc))
        self._h = h
        self._live = {}

    def submit(self, S: np.ndarray, Q: np.ndarray | None, select, eigs: bool = True) -> int:
        if not (S.flags.f_contiguous and S.dtype == np.float64):
            raise ValueError("S must be a Fortran-ordered float64 array")
        if Q is not None and not (Q.flags.f_contiguous and Q.dtype == np.float64):
            raise ValueError("Q must be a Fortran-ordered float64 array")
        n = int(S.shape[0])
        sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32).reshape(-1))
        if sel.size != n:
            raise ValueError("select must have n entries")
        wr = np.zeros(max(n, 1)) if eigs else None
        wi = np.zeros(max(n, 1)) if eigs else None
        t = load().gbr_server_submit(
            self._h, n, S.ctypes.data_as(_dp), max(n, 1),
            Q.ctypes.data_as(_dp) if Q is not None else None, max(n, 1),
            sel.ctypes.data_as(_ip), wr.ctypes.data_as(_dp) if eigs else None,
            wi.ctypes.data_as(_dp) if eigs else None)
        if t < 0:
            raise GbrError(int(t), status_string(int(t)))
        self._live[t] = (S, Q, sel, wr, wi)
        return int(t)

    def _result(self, t, rc, st, m):
        if rc != 1:
            return None
        S, Q, sel, wr, wi = self._live.pop(t)
        n = S.shape[0]
        e = (wr[:n] + 1j * wi[:n]) if wr is not None else None
        return ReorderResult(status=st.value, m=m.value, eigs=e, stats=None)

    def poll(self, ticket: int):
        st, m = ctypes.c_int(0), ctypes.c_int(0)
        rc = load().gbr_server_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(m))
        if rc < 0:
            raise KeyError(ticket)
        return self._result(ticket, rc, st, m)

    def wait(self, ticket: int, timeout_ms: int = -1):
        st, m = ctypes.c_int(0), ctypes.c_int(0)
        rc = load().gbr_server_wait(self._h, ticket, ctypes.byref(st), ctypes.byref(m),
                                    int(timeout_ms))
        if rc < 0:
            raise KeyError(ticket)
        return self._result(ticket, rc, st, m)

    def stats(self) -> dict:
        s = GbrServerStats()
        load().gbr_server_get_stats(self._h, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in GbrServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gbr_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
