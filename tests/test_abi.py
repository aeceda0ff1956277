"""The C-ABI library: builds for sm_103a, exports every symbol the header
declares, and checks its arguments before touching the GPU (these calls run
without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1905_04975_gb300 as g
from paper_1905_04975_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return g.load()


def header_functions():
    with open(os.path.join(ROOT, "include", "gbreorder.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbr_\w+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert "gbr_reorder" in names and "gbr_reorder_host" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in the header but not exported"
        assert name in g.SYMBOLS, f"{name} not bound in the Python layer"


def test_defaults_and_strings(lib):
    o = g.default_opts()
    assert (o.window, o.chain, o.precision, o.strong_test, o.validate, o.timing) == (128, 64, 2, 1, 1, 0)
    assert lib.gbr_version() >= 100
    for code in (0, 3, -1, -2, -3, -5, -6, -10, g.ERR_CUDA, g.ERR_NOMEM, g.ERR_TIMEOUT,
                 g.ERR_UNSUPPORTED):
        assert lib.gbr_status_string(code)


def test_error_codes_match_header(lib):
    """Every GBR_ERR_* of the header has the same value in the binding and a
    status string of its own."""
    with open(os.path.join(ROOT, "include", "gbreorder.h")) as f:
        codes = dict(re.findall(r"#define GBR_ERR_(\w+)\s+\((-\d+)\)", f.read()))
    assert "CAPTURING" in codes and len(codes) >= 7
    fallback = lib.gbr_status_string(-999)
    strings = set()
    for name, value in codes.items():
        assert getattr(g, "ERR_" + name) == int(value), name
        s = lib.gbr_status_string(int(value))
        assert s and s != fallback, name
        strings.add(s)
    assert len(strings) == len(codes)


def call(lib, n, S, ldS, Q, ldQ, sel, opts=None):
    wr = np.zeros(max(n, 1))
    wi = np.zeros(max(n, 1))
    m = ctypes.c_int(-7)
    st = g.GbrStats()
    o = opts or g.default_opts()
    rc = lib.gbr_reorder(n, S, ldS, Q, ldQ,
                         sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if sel is not None else None,
                         wr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         wi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(m),
                         ctypes.byref(o), ctypes.byref(st), None)
    return rc, m.value


def test_argument_errors_before_gpu(lib):
    dummy = ctypes.c_void_p(0x1000)  # never dereferenced: argument checks come first
    sel = np.zeros(8, np.int32)
    assert call(lib, -1, dummy, 8, None, 8, sel)[0] == -1
    assert call(lib, 8, None, 8, None, 8, sel)[0] == -2
    assert call(lib, 8, dummy, 7, None, 8, sel)[0] == -3
    assert call(lib, 8, dummy, 8, dummy, 4, sel)[0] == -5
    assert call(lib, 8, dummy, 8, None, 8, None)[0] == -6
    bad = g.default_opts()
    bad.window = 300
    assert call(lib, 0, None, 1, None, 1, sel, bad)[0] == -10
    bad = g.default_opts()
    bad.chain = 127
    assert call(lib, 0, None, 1, None, 1, sel, bad)[0] == -10
    ozk = g.default_opts()
    ozk.precision = 7
    assert call(lib, 0, None, 1, None, 1, sel, ozk)[0] == g.ERR_UNSUPPORTED
    # n = 0 is a no-op that succeeds without a GPU
    rc, m = call(lib, 0, None, 1, None, 1, sel)
    assert rc == 0 and m == 0
    # windows above 128: persistent schedule with FP64 updates only
    for prec in (g.PREC_FMA, g.PREC_DMMA):
        wide = g.make_opts(window=256, chain=128, precision=prec)
        assert call(lib, 0, None, 1, None, 1, sel, wide)[0] == 0
    wide = g.make_opts(window=256, chain=128, precision="ozaki")
    assert call(lib, 0, None, 1, None, 1, sel, wide)[0] == g.ERR_UNSUPPORTED
    wide = g.make_opts(window=200, chain=100, sched="sequential")
    assert call(lib, 0, None, 1, None, 1, sel, wide)[0] == g.ERR_UNSUPPORTED
    bad = g.default_opts()
    bad.window, bad.chain = 257, 64
    assert call(lib, 0, None, 1, None, 1, sel, bad)[0] == -10


def test_update_panel_argument_checks(lib):
    """gbr_update_panel checks its arguments (LAPACK-style -i) before any GPU
    work; rows = 0 is a no-op."""
    d = ctypes.c_void_p(0x1000)  # never dereferenced
    up = lib.gbr_update_panel
    assert up(-1, 8, d, 1, 8, d, 8, g.PREC_DMMA, None) == -1
    assert up(4, 0, d, 1, 8, d, 8, g.PREC_DMMA, None) == -2
    assert up(4, 129, d, 1, 8, d, 129, g.PREC_DMMA, None) == -2
    assert up(4, 8, None, 1, 8, d, 8, g.PREC_DMMA, None) == -3
    assert up(4, 8, d, 2, 8, d, 8, g.PREC_DMMA, None) == -4   # neither stride is 1
    assert up(4, 8, d, 0, 1, d, 8, g.PREC_DMMA, None) == -4
    assert up(4, 8, d, 1, 8, None, 8, g.PREC_DMMA, None) == -6
    assert up(4, 8, d, 1, 8, d, 7, g.PREC_DMMA, None) == -7
    assert up(4, 8, d, 1, 8, d, 8, 5, None) == -8
    assert up(0, 8, None, 1, 8, d, 8, g.PREC_OZAKI, None) == 0


def test_eigenvectors_argument_checks(lib):
    """gbr_eigenvectors checks its arguments before any GPU work; n = 0 is a
    no-op with m = 0."""
    d = ctypes.c_void_p(0x1000)  # never dereferenced
    ev = lib.gbr_eigenvectors
    m = ctypes.c_int(7)
    assert ev(-1, d, 4, None, 4, None, d, 4, ctypes.byref(m), None, None, None) == -1
    assert ev(4, None, 4, None, 4, None, d, 4, ctypes.byref(m), None, None, None) == -2
    assert ev(4, d, 3, None, 4, None, d, 4, ctypes.byref(m), None, None, None) == -3
    assert ev(4, d, 4, d, 3, None, d, 4, ctypes.byref(m), None, None, None) == -5
    assert ev(4, d, 4, None, 4, None, d, 3, ctypes.byref(m), None, None, None) == -8
    assert ev(0, None, 1, None, 1, None, None, 1, ctypes.byref(m), None, None, None) == 0
    assert m.value == 0


def test_reorder_gen_argument_checks(lib):
    """gbr_reorder_gen checks its arguments before any GPU work; options
    the pair path does not build (split precision off the persistent
    schedule, other slice counts) are refused; n = 0 is a no-op."""
    d = ctypes.c_void_p(0x1000)  # never dereferenced
    sel = np.zeros(4, dtype=np.int32)
    ip = sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    m = ctypes.c_int(7)
    seq = g.make_opts(sched="sequential")

    def call(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, sel_p, opts):
        return lib.gbr_reorder_gen(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, sel_p, None, None,
                                   ctypes.byref(m), ctypes.byref(opts) if opts else None, None, None)

    assert call(-1, d, 4, d, 4, None, 4, None, 4, ip, seq) == -1
    assert call(4, d, 4, None, 4, None, 4, None, 4, ip, seq) == -2
    assert call(4, d, 3, d, 4, None, 4, None, 4, ip, seq) == -3
    assert call(4, d, 4, d, 3, None, 4, None, 4, ip, seq) == -3
    assert call(4, d, 4, d, 4, d, 3, None, 4, ip, seq) == -5
    assert call(4, d, 4, d, 4, None, 4, d, 2, ip, seq) == -5
    assert call(4, d, 4, d, 4, None, 4, None, 4, None, seq) == -6
    assert call(4, d, 4, d, 4, None, 4, None, 4, ip, g.make_opts(window=16, chain=15,
                                                                  sched="sequential")) == -10
    assert call(4, d, 4, d, 4, None, 4, None, 4, ip, g.make_opts(precision="ozaki",
                                                                  sched="sequential")) == g.ERR_UNSUPPORTED
    assert call(4, d, 4, d, 4, None, 4, None, 4, ip, g.make_opts(precision="ozaki",
                                                                  slices=5)) == g.ERR_UNSUPPORTED
    assert call(0, None, 1, None, 1, None, 1, None, 1, None, None) == 0
    assert m.value == 0


def test_qr_sweep_argument_checks(lib):
    """gbr_qr_sweep checks its arguments before any GPU work."""
    d = ctypes.c_void_p(0x1000)  # never dereferenced
    dp = ctypes.POINTER(ctypes.c_double)
    re = np.array([0.5, 0.5, 1.0, 2.0])
    im = np.array([0.3, -0.3, 0.0, 0.0])
    bad_im = np.array([0.3, 0.3, 0.0, 0.0])
    R, I, B = (a.ctypes.data_as(dp) for a in (re, im, bad_im))
    o = g.default_opts()

    def call(n, H, ldH, Q, ldQ, ns, r, i, opts=o):
        return lib.gbr_qr_sweep(n, H, ldH, Q, ldQ, ns, r, i,
                                ctypes.byref(opts) if opts is not None else None, None, None)

    assert call(-1, d, 4, None, 4, 4, R, I) == -1
    assert call(4, None, 4, None, 4, 4, R, I) == -2
    assert call(4, d, 3, None, 4, 4, R, I) == -3
    assert call(4, d, 4, d, 3, 4, R, I) == -5
    assert call(4, d, 4, None, 4, 3, R, I) == -6
    assert call(4, d, 4, None, 4, 4, R, B) == -6
    assert call(4, d, 4, None, 4, 4, None, I) == -6
    assert call(4, d, 4, None, 4, 4, R, I, g.make_opts(window=2)) == -10
    assert call(4, d, 4, None, 4, 4, R, I, g.make_opts(window=4)) == -10  # no room to move
    assert call(4, d, 4, None, 4, 4, R, I, g.make_opts(precision="ozaki")) == g.ERR_UNSUPPORTED
    assert call(2, d, 2, None, 2, 4, R, I) == 0     # n < 3: nothing to do
    assert call(0, None, 1, None, 1, 0, None, None, None) == 0


def batch_create(lib, count, n, S, ldS, Q, ldQ, sel, opts=None, want_out=True):
    ip = ctypes.POINTER(ctypes.c_int)
    arr = lambda a: a.ctypes.data_as(ip) if a is not None else None
    h = ctypes.c_void_p(None)
    o = opts or g.default_opts()
    st = np.zeros(max(count, 1), dtype=np.int32)
    return lib.gbr_batch_create(count, arr(n), S, arr(ldS), Q, arr(ldQ), arr(sel), ctypes.byref(o),
                                arr(st), ctypes.byref(h) if want_out else None, None)


def test_batched_argument_checks(lib):
    """Argument errors of the batched entry point come back before any GPU
    work (LAPACK-style -i)."""
    n = np.array([4, 6], dtype=np.int32)
    ld = np.array([4, 6], dtype=np.int32)
    fake = (ctypes.c_void_p * 2)(0x1000, 0x2000)
    sel = np.zeros(10, dtype=np.int32)
    assert batch_create(lib, -1, n, fake, ld, None, None, sel) == -1
    assert batch_create(lib, 2, None, fake, ld, None, None, sel) == -2
    assert batch_create(lib, 2, np.array([4, -1], np.int32), fake, ld, None, None, sel) == -2
    assert batch_create(lib, 2, n, None, ld, None, None, sel) == -3
    assert batch_create(lib, 2, n, (ctypes.c_void_p * 2)(0x1000, None), ld, None, None, sel) == -3
    assert batch_create(lib, 2, n, fake, np.array([4, 5], np.int32), None, None, sel) == -4
    assert batch_create(lib, 2, n, fake, ld, fake, None, sel) == -6
    assert batch_create(lib, 2, n, fake, ld, fake, np.array([4, 2], np.int32), sel) == -6
    assert batch_create(lib, 2, n, fake, ld, None, None, None) == -7
    assert batch_create(lib, 2, n, fake, ld, None, None, sel, want_out=False) == -10
    assert batch_create(lib, 2, n, fake, ld, None, None, sel, opts=g.make_opts(window=200)) == -8
    assert batch_create(lib, 2, n, fake, ld, None, None, sel, opts=g.make_opts(window=16, chain=15)) == -8
    assert batch_create(lib, 2, n, fake, ld, None, None, sel,
                        opts=g.make_opts(sched="sequential")) == g.ERR_UNSUPPORTED
    assert lib.gbr_batch_run(None, None, None, None, None, None, None) == -1
    lib.gbr_batch_destroy(None)  # no-op
    assert lib.gbr_status_string(g.ERR_PLAN_MISMATCH)


def test_tuner_defaults_without_tuning(lib):
    w, m, t, tuned = g.tune_get(300)
    assert not tuned and (w, m) == (128, 64) and t >= 64
    assert lib.gbr_autotune(0, 10, None) == -1
    assert lib.gbr_autotune(64, 0, None) == -2


def test_server_argument_checks(lib):
    cfg = g.GbrServerCfg()
    lib.gbr_server_default_cfg(ctypes.byref(cfg))
    assert cfg.mem_cap_bytes == 60_000_000_000 and cfg.max_inflight >= 1 and cfg.sms == 0
    assert cfg.ring_entries >= 1024 and cfg.device == -1
    h = ctypes.c_void_p(None)
    assert lib.gbr_server_create(ctypes.byref(cfg), None) == -2
    bad = g.GbrServerCfg()
    lib.gbr_server_default_cfg(ctypes.byref(bad))
    bad.ring_entries = 10
    assert lib.gbr_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.ring_entries, bad.mem_cap_bytes = 1 << 20, 0
    assert lib.gbr_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.mem_cap_bytes, bad.sms = 1 << 30, -1
    assert lib.gbr_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.sms = 0
    bad.opts.sched = g.SCHED_SEQUENTIAL
    assert lib.gbr_server_create(ctypes.byref(bad), ctypes.byref(h)) == g.ERR_UNSUPPORTED
    assert lib.gbr_server_submit(None, 4, None, 4, None, 4, None, None, None) == -1
    assert lib.gbr_server_poll(None, 0, None, None) == -1
    assert lib.gbr_server_wait(None, 0, None, None, 0) == -1
    assert lib.gbr_server_get_stats(None, None) == -1
    lib.gbr_server_destroy(None)


def test_struct_layouts_match_header(tmp_path):
    """Every public struct has the same size and field offsets in the C
    header (compiled with gcc) as in the Python binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"gbr_opts": g.GbrOpts, "gbr_stats": g.GbrStats, "gbr_ev_stats": g.GbrEvStats,
               "gbr_server_cfg": g.GbrServerCfg, "gbr_server_stats": g.GbrServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gbreorder.h"',
             'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = {}
    for ln in out.splitlines():
        cname, key, val = ln.split()
        seen[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert seen[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert seen[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_tune_table_json_round_trip(lib, tmp_path):
    """The autotuner table persists as JSON (host only, no GPU): a loaded
    table answers gbr_tune_get, saves back to the same classes, and invalid
    or malformed files change nothing."""
    src = tmp_path / "tune.json"
    src.write_text('{"tune": [\n  {"n_max": 32, "window": 32, "chain": 24, "tile": 64},\n'
                   '  {"n_max": 512, "window": 128, "chain": 64, "tile": 256}\n]}\n')
    assert g.tune_load(src) == 2
    assert g.tune_get(20)[:2] == (32, 24) and g.tune_get(20)[3]
    assert g.tune_get(300) == (128, 64, 256, True)
    out = tmp_path / "saved.json"
    assert g.tune_save(out) >= 2
    text = out.read_text()
    assert '"n_max": 32, "window": 32, "chain": 24, "tile": 64' in text
    assert '"n_max": 512, "window": 128, "chain": 64, "tile": 256' in text
    # reload what was saved: same answers
    assert g.tune_load(out) >= 2
    assert g.tune_get(300) == (128, 64, 256, True)
    for bad in ['{"tune": [{"n_max": 64, "window": 200, "chain": 64, "tile": 64}]}',
                '{"tune": [{"n_max": 64, "window": 64, "chain": 63, "tile": 64}]}',
                '{"tune": [{"n_max": 48, "window": 32, "chain": 16, "tile": 64}]}',
                '{"tune": [{"n_max": 64, "window": 32, "chain": 16, "tile": 100}]}',
                '{"tune": [{"n_max": 64, "window": 32, "tile": 64}]}',
                '{"other": 1}']:
        f = tmp_path / "bad.json"
        f.write_text(bad)
        with pytest.raises(g.GbrError) as ei:
            g.tune_load(f)
        assert ei.value.status == -3
    assert g.tune_get(300) == (128, 64, 256, True)  # unchanged
    with pytest.raises(g.GbrError):
        g.tune_load(tmp_path / "missing.json")
    assert lib.gbr_tune_load(None) == -1 and lib.gbr_tune_save(None) == -1
