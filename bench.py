#!/usr/bin/env python
"""Benchmark: selected eigenvalues reordered per second on one GB300.

Workload (default): a real Schur form of order n = 16000 from the seeded
generator (60% of positions in 1x1 blocks, 40% in standardized 2x2 blocks,
N(0,1) strict upper part) with its eigenvalues in 20 tight clusters (spread
1e-6), Q = product of 64 seeded Householder reflectors, 50% of the
eigenvalues selected, window 128, chain 64.  The line's own fields are the
FP64 updates on the FMA pipe; `split_precision` holds the same workload with
split-precision updates on the tensor cores (both with the accuracy of one
result), `fp64_tensor_core` a shorter run with FP64 DMMA updates.

A step is one full reordering (every planner, window, update and eigenvalue
kernel of the call).  S and Q (4.1 GB, larger than L2) are restored from a
pristine device copy before each step, outside the timed region; that
rewrite also evicts them from L2.  Each step is timed with CUDA events on the
library's stream; `value` = selected eigenvalues of all steps (and ranks) /
summed step time.

Also reported:
  roofline      the dominant kernel's algorithmic work / its event-timed
                duration inside the timed steps, against the measured peak;
  e2e           the same metric through gbr_reorder_host (pinned host
                buffers, H2D + D2H inside the timed region);
  cpu_baseline  the CPU oracle on a bounded sample of the same workload;
  clocks        nvidia-smi samples taken during the timed region.

`--impl reference` times the CPU oracle instead (rank 0 only).
Multi-GPU: one reordering does not shard; N ranks run N independent
replicas (`scaling: weak`).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import schur_inputs as si  # noqa: E402

WORKLOADS = {
    "n4000": dict(name="n4000", n=4000, select=0.35, q="64 Householder reflectors", window=128,
                  chain=64),
    # n = 400 is latency bound (a few chains of window tasks): the smaller
    # window measured fastest for it (window sweep on the GPU: 6.26 ms per
    # step at w = 32, m = 16 against 8.09 ms at 128, 64)
    "n400": dict(name="n400", n=400, select=0.30, q="identity", window=32, chain=16),
    "n16000c": dict(name="n16000c", n=16000, select=0.50, q="64 Householder reflectors",
                    window=128, chain=64, clusters="20 clusters, spread 1e-6"),
    "batch4096": dict(name="batch4096", kind="batch", count=4096, nmin=32, nmax=512,
                      select="U(0.2, 0.6) per instance", q="min(n, 64) Householder reflectors"),
    "eigvec4000": dict(name="eigvec4000", kind="eigvec", n=4000, select=0.35,
                       q="64 Householder reflectors", window=128, chain=64),
    "serve": dict(name="serve", kind="serve", nmin=64, nmax=8192, select="U(0.1, 0.6)",
                  q="8 Householder reflectors", mem_cap=60e9),
    "g4000": dict(name="g4000", kind="gen", n=4000, select=0.35,
                  q="Q and Z: 64 Householder reflectors each", window=64, chain=32),
    "h4000": dict(name="h4000", kind="sweep", n=4000, shifts=64,
                  q="64 Householder reflectors", window=64, chain=16),
}
SWEEP_METRIC = "shifts chased per second (one bulge-chasing sweep)"

# FP64 on the FMA pipe: 2 fused multiply-adds per clock per SM (the nominal
# 1.25 TFLOP/s FP64 rate of the part), 152 SMs, 2070 MHz maximum SM clock.
FP64_FMA_PEAK = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_FMA_PEAK_SOURCE = ("FP64 FMA: 2 per clock per SM x 152 SMs x 2070 MHz x 2 flops "
                        "(nominal FP64 1.25 TFLOP/s); measured DFMA probe 1.195 TFLOP/s")
METRIC = "selected eigenvalues reordered per second"

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the current kernels (the sched_kernel captures under profiles/);
# a workload has no entry while no capture of the current build exists (g4000:
# its pass now runs as three chunked launches, the capture was of one launch).
NCU_TRAFFIC = {("n4000", "dmma"): 1.937360e9 + 2.652817e9,
               ("n4000", "fma"): 1.299070e9 + 2.728422e9,
               ("n4000", "ozaki"): 2.886808e9 + 4.348523e9,
               ("eigvec4000", "evgemm"): 1.052943e9 + 0.125283e9,
               ("h4000", "persistent-dmma"): 0.220709e9 + 0.187885e9}


def f_min_flops(n, swaps):
    """The unblocked scalar floor of a reordering: every adjacent swap applied
    as a rotation to two rows and two columns of S and two columns of Q, 6
    flops per element pair over about 2n elements, i.e. 12 n flops per swap
    (about 6 p (1 - p) n^3 in all for a fraction p selected)."""
    return 12.0 * n * swaps


def whole_job_rate(units, local_ms, dist=None, device="cpu"):
    """Replicas: every rank processed `units` in `local_ms`; the job's time is
    the slowest rank's (max over ranks), and its rate is all ranks' units over
    that time.  Returns (rate per second, job time in ms)."""
    world = 1
    job_ms = float(local_ms)
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([job_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        job_ms = float(t.item())
    return units * world / (job_ms / 1e3), job_ms


def fp64_roof_basis(prec, pk, src):
    """(tile name, bound, peak TFLOP/s, peak source) of the FP64 update tiles
    of a precision: FMA-pipe tiles against the FP64 FMA rate, DMMA tiles
    against the FP64 tensor rate (measured bf16 peak x nominal ratio)."""
    if prec == "fma":
        return "FP64 FMA tiles", "alu", FP64_FMA_PEAK, FP64_FMA_PEAK_SOURCE
    return ("DMMA tiles", "tensor", pk["bf16_tflops"] * (1.25 / 2250.0),
            f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 1.25/2250 "
            "(FP64 DMMA probe: 1.047 TF/s)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def make_inputs(wl, seed=0):
    return si.config("n4000" if wl["name"] == "eigvec4000" else wl["name"], seed)


def block_list(S, sel):
    """Diagonal blocks of S: starts, sizes and per-block selection (a 2x2
    block is selected if either position is)."""
    n = S.shape[0]
    sub = np.append(np.diag(S, -1) != 0, False)
    starts, sizes = [], []
    p = 0
    while p < n:
        sz = 2 if sub[p] else 1
        starts.append(p)
        sizes.append(sz)
        p += sz
    selb = [bool(sel[s] or (sz == 2 and sel[s + 1])) for s, sz in zip(starts, sizes)]
    return starts, sizes, selb


def first_selected(n, starts, sizes, selb, k):
    """Selection of the first k selected blocks (top to bottom)."""
    sub_sel = np.zeros(n, np.int32)
    taken = 0
    for s, sz, flag in zip(starts, sizes, selb):
        if flag and taken < k:
            sub_sel[s:s + sz] = 1
            taken += 1
    return sub_sel


def swaps_needed(selb, k_blocks):
    """Adjacent block swaps of the stable partition of the first k selected
    blocks (each passes every unselected block above it)."""
    cnt, unsel_above, taken = 0, 0, 0
    for flag in selb:
        if flag:
            if taken >= k_blocks:
                break
            cnt += unsel_above
            taken += 1
        else:
            unsel_above += 1
    return cnt


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def calibrate_sample(S, sel, run, budget_s):
    """Grows k (the first k selected blocks) until run(sub_sel) takes about
    budget_s / 3.  Returns (k, result, seconds)."""
    n = S.shape[0]
    starts, sizes, selb = block_list(S, sel)
    nsel_blocks = sum(selb)
    k = max(1, nsel_blocks // 64)
    while True:
        sub_sel = first_selected(n, starts, sizes, selb, k)
        t0 = time.perf_counter()
        r = run(sub_sel)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or k >= nsel_blocks:
            return k, r, dt
        k = min(nsel_blocks, int(k * 1.6) + 1)


def sample_record(S, sel, k, dt, nswaps, cores, what, who):
    """A timed sample of the first k selected blocks in the metric's unit:
    the eigenvalue-equivalent work it did (the workload's selected
    eigenvalues x its share of the workload's adjacent block swaps) over
    the time it took."""
    n = S.shape[0]
    starts, sizes, selb = block_list(S, sel)
    nsel_blocks = sum(selb)
    full_swaps = swaps_needed(selb, nsel_blocks)
    nsel = int(np.sum([sz for sz, f in zip(sizes, selb) if f]))
    share = nswaps / max(full_swaps, 1)
    est_full = dt / max(share, 1e-300)
    return {"value": nsel * share / dt, "unit": "eigs/s", "cores": cores, "kind": "oracle",
            "secs": dt, "est_full_s": est_full, "k": k,
            "sample": (f"{who}: first {k} of {nsel_blocks} selected blocks of the n={n} {what} "
                       f"({nswaps} of {full_swaps} block swaps) in {dt:.2f} s on {cores} "
                       f"core(s); value = the eigenvalue-equivalent share of the workload done "
                       f"(swaps) per second (whole workload est. {est_full:.0f} s)")}


def cpu_oracle_sample(S, Q, sel, budget_s=15.0, run=None, what="workload", k=None, lib=None,
                      cores=1, who="oracle, 1 thread"):
    """The oracle on the first k selected blocks (top to bottom) of the
    workload; k grown until ~budget_s / 3 of work unless given.  run(sub_sel)
    runs the oracle and returns its result dict (default: the standard-form
    reordering of (S, Q) with the oracle library `lib`)."""
    import oracle
    if run is None:
        run = lambda sub_sel: oracle.reorder(S, Q, sub_sel, lib=lib)
    if k is None:
        k, r, dt = calibrate_sample(S, sel, run, budget_s)
    else:
        n = S.shape[0]
        starts, sizes, selb = block_list(S, sel)
        sub_sel = first_selected(n, starts, sizes, selb, k)
        t0 = time.perf_counter()
        r = run(sub_sel)
        dt = time.perf_counter() - t0
    return sample_record(S, sel, k, dt, r["nswaps"], cores, what, who)


def dtrsen_sample(S, Q, sel, k, cores):
    """LAPACK dtrsen (scipy, called, not read) on the same first k selected
    blocks, Q accumulated, no condition numbers; BLAS threads = cores."""
    from scipy.linalg import lapack
    n = S.shape[0]
    starts, sizes, selb = block_list(S, sel)
    sub_sel = first_selected(n, starts, sizes, selb, k)
    St, Qt = np.asfortranarray(S.copy()), np.asfortranarray(Q.copy())
    t0 = time.perf_counter()
    out = lapack.dtrsen(sub_sel, St, Qt, job="N", wantq=1, overwrite_t=1, overwrite_q=1,
                        lwork=max(1, n), liwork=1)
    dt = time.perf_counter() - t0
    info = out[-1]
    rec = sample_record(S, sel, k, dt, swaps_needed(selb, k), cores, "workload",
                        "scipy LAPACK dtrsen (OpenBLAS)")
    rec["kind"] = "library"
    rec["info"] = int(info)
    return rec


def cpu_leg(wl, budget_s=15.0):
    """The CPU baselines of a reordering workload, in a process of their own
    (no torch): the oracle single-threaded, the same oracle built with
    OpenMP on all host cores, and scipy's dtrsen, on the same bounded
    sample (the first k selected blocks).  Prints one JSON object."""
    import oracle
    if wl.get("kind") == "batch":
        print(json.dumps(batch_cpu_sample(batch_inputs(wl), budget_s=budget_s)), flush=True)
        return 0
    S, Q, sel = make_inputs(wl)
    cores = host_cores()
    one = cpu_oracle_sample(S, Q, sel, budget_s=budget_s, lib=oracle.load())
    k = one["k"]
    omp = cpu_oracle_sample(S, Q, sel, k=k, lib=oracle.load_omp(), cores=cores,
                            who=f"oracle, OpenMP {cores} threads")
    lap = dtrsen_sample(S, Q, sel, k, cores)
    best = omp if omp["value"] >= one["value"] else one
    out = dict(best)
    out.update({"cpu_model": cpu_model(), "host_cores": cores,
                "single_thread": one, "openmp": omp, "scipy_dtrsen": lap})
    print(json.dumps(out), flush=True)
    return 0


def run_cpu_leg(wl):
    """Runs cpu_leg in a fresh interpreter (OpenMP and BLAS threads on all
    host cores, nothing else running); returns its JSON object or an error
    record."""
    cores = host_cores()
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores))
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload",
                        wl["name"]], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        return {"error": p.stderr[-500:]}
    return json.loads(p.stdout.strip().splitlines()[-1])


def reference_reorder_steps(args, S, Q, sel, what, run_one, budget_s, cores, who):
    """Reference-arm steps: each one the oracle on the same bounded sample
    (k calibrated once, untimed), timed as it runs.  Returns (value,
    ms_per_step, last record)."""
    k, _, _ = calibrate_sample(S, sel, run_one, budget_s)
    recs = []
    for i in range(args.warmup + args.steps):
        rec = cpu_oracle_sample(S, Q, sel, k=k, run=run_one, what=what, cores=cores, who=who)
        if i >= args.warmup:
            recs.append(rec)
    secs = sum(r["secs"] for r in recs)
    units = sum(r["value"] * r["secs"] for r in recs)
    return units / secs, 1e3 * secs / len(recs), recs[-1]


def reference_instances(args, probs, budget_s):
    """Reference-arm steps for independent instances (batch, serving): each
    step the oracle on the same first instances (count calibrated once),
    one instance per worker process on all host cores."""
    cores = host_cores()
    with InstancePool(cores) as pool:
        count = pool.calibrate(probs, budget_s)
        recs = []
        for i in range(args.warmup + args.steps):
            rec = pool.sample(probs, count)
            if i >= args.warmup:
                recs.append(rec)
    secs = sum(r["secs"] for r in recs)
    value = sum(r["value"] * r["secs"] for r in recs) / secs
    return value, 1e3 * secs / len(recs), recs[-1]


def run_reference(args, wl):
    """The reference arm: the CPU oracle (the reference is a paper, with no
    program of its own), its OpenMP build on all host cores, on a bounded
    sample of the workload per step.  ms_per_step is the time of the
    sample actually run; the whole workload's estimated time is reported
    under its own key."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cores = host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    lib = oracle.load_omp()
    extra = {}
    if wl.get("kind") == "serve":
        reqs = si.request_stream(args.requests, seed=2000, nmin=wl["nmin"], nmax=wl["nmax"],
                                 pmin=0.1, pmax=0.6)
        # the oracle's cost grows as n^3: its sample takes the requests of
        # order <= 1024 of the stream, in order
        probs = [si.serve_problem(n, p, sd) for _, n, p, sd in reqs if n <= 1024][:200]
        cfg = {"workload": "serve", "n": "requests of order <= 1024 of the stream",
               "select": wl["select"], "q": wl["q"]}
        value, ms, rec = reference_instances(args, probs, budget_s=4.0)
        unit, metric = "eigs/s", METRIC
    elif wl.get("kind") == "eigvec":
        S, Q, _ = make_inputs(wl)
        n = S.shape[0]
        recs = []
        for i in range(args.warmup + args.steps):
            cb = eigvec_cpu_sample(S, Q)
            if i >= args.warmup:
                recs.append(cb)
        secs = sum(r["secs"] for r in recs)
        value = sum(r["value"] * r["secs"] for r in recs) / secs
        ms, rec = 1e3 * secs / len(recs), recs[-1]
        unit, metric = "eigenvectors/s", "eigenvectors computed per second"
        cfg = {"workload": wl["name"], "n": n, "eigenvectors": f"all ({n})", "q": wl["q"]}
    elif wl.get("kind") == "sweep":
        H, Q, sh = si.sweep_config(wl["name"])
        recs = []
        for i in range(args.warmup + args.steps):
            cb = sweep_cpu(H, Q, sh)
            if i >= args.warmup:
                recs.append(cb)
        secs = sum(r["secs"] for r in recs)
        value = sum(r["value"] * r["secs"] for r in recs) / secs
        ms, rec = 1e3 * secs / len(recs), recs[-1]
        unit, metric = "shifts/s", SWEEP_METRIC
        cfg = {"workload": wl["name"], "n": wl["n"], "shifts": wl["shifts"], "q": wl["q"],
               "window": wl["window"], "chain": wl["chain"]}
    elif wl.get("kind") == "gen":
        S, T, Q, Z, sel = si.gen_config(wl["name"])
        run_one = lambda ss: oracle.gen_reorder(S, T, Q, Z, ss)
        value, ms, rec = reference_reorder_steps(args, S, Q, sel, "pair workload", run_one, 4.0,
                                                 1, "generalized oracle, 1 thread")
        unit, metric = "eigs/s", METRIC
        cfg = {"workload": wl["name"], "n": wl["n"], "select": wl["select"], "q": wl["q"],
               "window": wl["window"], "chain": wl["chain"]}
    elif wl.get("kind") == "batch":
        probs = batch_inputs(wl)
        cfg = {"workload": wl["name"], "instances": wl["count"],
               "n": f"U{{{wl['nmin']}..{wl['nmax']}}}", "select": wl["select"], "q": wl["q"]}
        value, ms, rec = reference_instances(args, probs, budget_s=4.0)
        unit, metric = "eigs/s", METRIC
    else:
        S, Q, sel = make_inputs(wl)
        run_one = lambda ss: oracle.reorder(S, Q, ss, lib=lib)
        value, ms, rec = reference_reorder_steps(args, S, Q, sel, "workload", run_one, 4.0,
                                                 cores, f"oracle, OpenMP {cores} threads")
        unit, metric = "eigs/s", METRIC
        cfg = {"workload": wl["name"], "n": wl["n"], "select": wl["select"],
               "q": wl["q"], "window": wl["window"], "chain": wl["chain"]}
        extra["estimated_full_workload_ms"] = 1e3 * rec["est_full_s"]
    cb = {k2: v for k2, v in rec.items() if k2 not in ("secs", "est_full_s", "k")}
    cb["value"] = value
    cb["cpu_model"] = cpu_model()
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


def expected_selected(S, sel):
    n = S.shape[0]
    cnt = 0
    p = 0
    while p < n:
        if p + 1 < n and S[p + 1, p] != 0:
            cnt += 2 if (sel[p] or sel[p + 1]) else 0
            p += 2
        else:
            cnt += 1 if sel[p] else 0
            p += 1
    return cnt


def error_report(g, torch, S_np, Q_np, sel, S, Q, S0, Q0, opts, stream, with_oracle=True):
    """Accuracy of one reordering of the workload (after the timed steps):
    residual ||A - Q S Q^T||_F / ||A||_F and ||Q^T Q - I||_F estimated with 32
    Gaussian probe vectors on the GPU, eigenvalue order against the stable
    partition of the input eigenvalues, and for n <= 4000 the difference to
    the FP64 oracle's result (eigenvalues, leading invariant subspace)."""
    import oracle
    from tests.helpers import block_eigs, expected_order, is_standard, sin_angle
    with torch.cuda.stream(stream):
        S.copy_(S0)
        Q.copy_(Q0)
    stream.synchronize()
    r = g.reorder(S, Q, sel, opts=opts, stream=stream)
    stream.synchronize()
    n = S_np.shape[0]
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(n, 32, dtype=torch.float64, device="cuda", generator=gen)
    S0c, Q0c = S0.contiguous(), Q0.contiguous()
    Sc, Qc = S.contiguous(), Q.contiguous()
    AX = Q0c @ (S0c @ (Q0c.T @ X))
    res = (torch.linalg.norm(AX - Qc @ (Sc @ (Qc.T @ X))) / torch.linalg.norm(S0c)).item() / 32 ** 0.5
    orth = torch.linalg.norm(Qc.T @ (Qc @ X) - X).item() / 32 ** 0.5
    Sg = g.to_host(S)
    got = block_eigs(Sg)
    want, m = expected_order(S_np, sel)
    out = {"status": r.status, "residual_est": res, "orth_est": orth, "bound_50n_eps": 50 * n * 2.0 ** -52,
           "eig_order_max_rel_dev": float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)))}
    out["rejected"] = int(r.stats.rejected)
    out["standard_form"] = bool(is_standard(Sg))
    if n <= 4000 and with_oracle:
        t0 = time.perf_counter()
        ref = oracle.reorder(S_np, Q_np, sel)
        out["oracle_s"] = time.perf_counter() - t0
        oe = ref["wr"] + 1j * ref["wi"]
        out["vs_oracle_eig_max_rel_dev"] = float(np.max(np.abs(got - oe) / np.maximum(np.abs(oe), 1.0)))
        Qg = g.to_host(Q)
        out["vs_oracle_sin_angle"] = sin_angle(Qg[:, :m], ref["Q"][:, :m]) if 0 < m < n else 0.0
    return out


def batch_inputs(wl, seed=0):
    """The batched workload: per instance (S, Q, select) from the seeded
    generator, n ~ U{nmin..nmax}, p ~ U(0.2, 0.6)."""
    out = []
    for n, p, sd in si.batch_problems(wl["count"], seed, wl["nmin"], wl["nmax"]):
        out.append(si.reorder_problem(n, sd, select_frac=p, q="householder",
                                      reflectors=min(n, 64)))
    return out


def _oracle_instance(prob):
    """One instance through the oracle (a worker process of InstancePool)."""
    import oracle
    S, Q, sel = prob
    oracle.reorder(S, Q, sel)
    return int(expected_selected(S, sel))


def _pool_ready(_):
    import oracle
    oracle.load()
    return os.getpid()


class InstancePool:
    """The oracle over independent instances: in turn on one core
    (workers=1), or one instance per worker on `workers` processes started
    with spawn (and warmed up) before any timing."""

    def __init__(self, workers):
        self.workers = workers
        self.ex = None

    def __enter__(self):
        if self.workers > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            self.ex = ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"))
            list(self.ex.map(_pool_ready, range(4 * self.workers)))
        return self

    def __exit__(self, *a):
        if self.ex:
            self.ex.shutdown()

    def sample(self, probs, count):
        t0 = time.perf_counter()
        if self.ex is None:
            eigs = sum(_oracle_instance(p) for p in probs[:count])
        else:
            eigs = sum(self.ex.map(_oracle_instance, probs[:count], chunksize=1))
        dt = time.perf_counter() - t0
        who = "1 core" if self.ex is None else f"{self.workers} worker processes"
        return {"value": eigs / dt, "unit": "eigs/s", "cores": self.workers, "kind": "oracle",
                "secs": dt, "count": count,
                "sample": f"first {count} of {len(probs)} instances ({eigs} selected "
                          f"eigenvalues) in {dt:.2f} s on {who}"}

    def calibrate(self, probs, budget_s):
        """Instance count whose sample takes about budget_s."""
        count = min(len(probs), 2 * self.workers)
        while True:
            rec = self.sample(probs, count)
            if rec["secs"] >= budget_s / 2 or count >= len(probs):
                return count
            count = min(len(probs), int(count * budget_s / max(rec["secs"], 1e-3) * 0.8) + 1)


def batch_cpu_sample(probs, budget_s=12.0):
    """The oracle on the first instances of the batch: on one core until
    ~budget_s, then the same instances on all host cores (one instance per
    worker process).  The faster is the headline value; both are kept."""
    with InstancePool(1) as p1:
        count = p1.calibrate(probs, budget_s)
        one = p1.sample(probs, count)
    cores = host_cores()
    out = one
    if cores > 1:
        with InstancePool(cores) as pc:
            many = pc.sample(probs, count)
        out = dict(many if many["value"] > one["value"] else one)
        out["single_thread"] = one
        out["all_cores"] = many
    out["cpu_model"] = cpu_model()
    return out


def run_batch(args, wl):
    import torch
    import paper_1905_04975_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()
    probs = batch_inputs(wl, seed=rank)
    ns = [S.shape[0] for S, _, _ in probs]
    sizes = np.array([n * n for n in ns], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)])
    tot = int(off[-1])
    nsel = int(sum(expected_selected(S, sel) for S, _, sel in probs))
    # one flat pinned host buffer per matrix kind, column-major instances back to back
    hS = torch.empty(tot, dtype=torch.float64).pin_memory()
    hQ = torch.empty(tot, dtype=torch.float64).pin_memory()
    hSn, hQn = hS.numpy(), hQ.numpy()
    for i, (S, Q, _) in enumerate(probs):
        hSn[off[i]:off[i + 1]] = S.ravel(order="F")
        hQn[off[i]:off[i + 1]] = Q.ravel(order="F")
    dS, dQ = hS.cuda(), hQ.cuda()
    dS0, dQ0 = dS.clone(), dQ.clone()

    def views(buf):
        return [buf[off[i]:off[i + 1]].view(ns[i], ns[i]).t() for i in range(len(ns))]
    Sv, Qv = views(dS), views(dQ)
    sels = [sel for _, _, sel in probs]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    tuned = g.autotune(wl["nmax"], 256, stream=stream)
    tune_s = time.perf_counter() - t0
    choices = {c: g.tune_get(2 ** c) for c in range(5, 10)}
    opts = g.make_opts(window=g.AUTO, chain=g.AUTO, precision=args.precision, timing=True)
    t0 = time.perf_counter()
    batch = g.Batch(Sv, Qv, sels, opts=opts, stream=stream)
    plan_s = time.perf_counter() - t0

    def restore():
        with torch.cuda.stream(stream):
            dS.copy_(dS0)
            dQ.copy_(dQ0)
        stream.synchronize()

    def step():
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = batch.run(stream=stream)
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        r, _ = step()
        assert r.rc == 0 and np.all(r.status == 0), r.rc
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            r, t = step()
            ms.append(t)
            stats.append(r.stats)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    value, total_ms = whole_job_rate(nsel * args.steps, sum(ms), dist, "cuda")
    st0 = stats[0]
    ms_sched = sum(s.ms_sched for s in stats) / len(stats)
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)
    upd_iss = st0.upd_flops_issued if st0.upd_flops_issued > 0 else st0.upd_flops
    work = upd_iss + st0.win_flops
    achieved = work / (ms_sched / 1e3) / 1e12
    tname, bound, fpk, fsrc = fp64_roof_basis(args.precision, pk, src)
    roof = {"kernel": f"sched_kernel (persistent, all instances: window tasks + {tname})",
            "bound": bound, "achieved": achieved, "peak": fpk, "unit": "TFLOP/s",
            "frac": achieved / fpk, "traffic": None, "peak_source": fsrc,
            "flops_per_launch": work, "launches_per_step": 1, "avg_launch_ms": ms_sched,
            "share_of_step": ms_sched / (total_ms / args.steps),
            "critical_path_model_ms": st0.sched_cp_ms}

    # end to end: inputs from pinned host memory, results back, every step
    e2e = None
    if args.e2e_steps > 0:
        oS = torch.empty(tot, dtype=torch.float64).pin_memory()
        oQ = torch.empty(tot, dtype=torch.float64).pin_memory()
        et = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                dS.copy_(hS, non_blocking=True)
                dQ.copy_(hQ, non_blocking=True)
            rr = batch.run(stream=stream)
            with torch.cuda.stream(stream):
                oS.copy_(dS, non_blocking=True)
                oQ.copy_(dQ, non_blocking=True)
            stream.synchronize()
            dt = time.perf_counter() - t0
            assert rr.rc == 0
            if i > 0:
                et.append(dt)
        e2e = {"value": nsel * len(et) / sum(et) * world, "unit": "eigs/s",
               "h2d_bytes_per_step": 2 * tot * 8 + 4 * int(sum(ns)),
               "d2h_bytes_per_step": 2 * tot * 8 + 16 * int(sum(ns))}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = batch_cpu_sample(probs)
    batch.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "eigs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "instances": len(ns),
                           "n": f"U{{{wl['nmin']}..{wl['nmax']}}}", "select": wl["select"],
                           "selected_eigs": nsel, "q": wl["q"], "window": "autotuned",
                           "chain": "autotuned", "precision": args.precision,
                           "l2": f"S,Q ({2 * tot * 8 / 1e9:.1f} GB > L2) restored from a device "
                                 "copy before each step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": int(sum(s.launches for s in stats)),
                "detail": {"windows": int(st0.windows), "tasks": int(st0.tasks),
                           "swaps": int(st0.swaps), "upd_flops": st0.upd_flops,
                           "win_flops": st0.win_flops, "plan_s": plan_s, "autotune_s": tune_s,
                           "classes_tuned": tuned,
                           "tuned": {f"n<={2 ** c}": v[:3] for c, v in choices.items()},
                           "host_graph_ms": st0.ms_graph, "host_order_ms": st0.ms_order}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _serve_make_pinned(n, p, sd):
    """One serving request in pinned host memory: the generator's row-major
    form of the request, copied transposed (torch's blocked CPU transpose)
    into pinned buffers whose memory is the column-major matrix."""
    import torch
    S, Q, sel = si.serve_problem(n, p, sd, order="C")
    nn = S.shape[0]
    tS = torch.empty((nn, nn), dtype=torch.float64).pin_memory()
    tQ = torch.empty((nn, nn), dtype=torch.float64).pin_memory()
    tS.copy_(torch.from_numpy(S).t())
    tQ.copy_(torch.from_numpy(Q).t())
    return tS, tQ, sel, int(expected_selected(S, sel))


class RequestFeed:
    """Serving requests generated ahead of their arrival by a pool of host
    threads (the generator's bulk work, random fills, matrix products and
    copies, runs without the interpreter lock), at most `ahead` in flight,
    in stream order."""

    def __init__(self, specs, workers, ahead=24, make=None):
        from concurrent.futures import ThreadPoolExecutor
        self.make = make or (lambda n, p, sd: si.serve_problem(n, p, sd))
        self.specs = specs
        self.ex = ThreadPoolExecutor(workers)
        self.futs = []
        self.next = 0
        self.ahead = ahead
        self._fill()

    def _fill(self):
        while self.next < len(self.specs) and len(self.futs) < self.ahead:
            n, p, sd = self.specs[self.next]
            self.futs.append(self.ex.submit(self.make, n, p, sd))
            self.next += 1

    def get(self):
        f = self.futs.pop(0)
        self._fill()
        return f.result()

    def close(self):
        self.ex.shutdown(cancel_futures=True)


def run_serve(args, wl):
    """Serving: a Poisson stream of requests (n log-uniform, see the
    workload) through the continuous-batching server.  A saturation burst
    first measures the throughput; the stream then arrives at each --load
    fraction of it.  Every request is an independent form from the seeded
    generator, made by host threads ahead of its arrival."""
    import torch
    import paper_1905_04975_gb300 as g

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    g.load()
    workers = max(1, min(8, host_cores() // 2))

    def specs(count, seed):
        return [(n, p, sd) for _, n, p, sd in
                si.request_stream(count, seed=seed, nmin=wl["nmin"], nmax=wl["nmax"],
                                  pmin=0.1, pmax=0.6, rate=1.0)]

    def run(rate, count, seed):
        """Submits `count` requests (Poisson arrivals at `rate` per second,
        or all at once when rate is None) and waits for all of them."""
        feed = RequestFeed(specs(count, seed), workers, make=_serve_make_pinned)
        srv = g.Server(mem_cap_bytes=wl["mem_cap"], precision=args.precision)
        late = 0.0
        try:
            gaps = np.random.default_rng(seed + 7).exponential(1.0 / rate, count) if rate else None
            pending = {}
            eigs = 0
            with ClockSampler(local) as clk:
                t0 = time.perf_counter()
                t_next = t0
                for i in range(count):
                    tS, tQ, sel, nsel_i = feed.get()
                    item = (tS, tQ, tS.numpy().T, tQ.numpy().T)   # Fortran-ordered views
                    if gaps is not None:
                        t_next += gaps[i]
                        dt = t_next - time.perf_counter()
                        if dt > 0:
                            time.sleep(dt)
                        else:
                            late = max(late, -dt)
                    t = srv.submit(item[2], item[3], sel, eigs=False)
                    pending[t] = item
                    eigs += nsel_i
                    for tk in [tk for tk in pending if srv.poll(tk) is not None]:
                        del pending[tk]
                for tk in list(pending):
                    r = srv.wait(tk, -1)
                    assert r.status >= 0, r.status
                wall = time.perf_counter() - t0
            st = srv.stats()
        finally:
            srv.close()
            feed.close()
        return st, wall, eigs, clk.summary(), late

    burst = max(20, args.requests // 10)
    st_b, wall_b, eigs_b, clk_b, _ = run(None, burst, 1000 + rank)
    sat = st_b["req_per_s"]
    loads = []
    for li, load in enumerate(args.loads):
        st, wall, eigs, clk, late = run(load * sat, args.requests, 2000 + 100 * li + rank)
        loads.append({"load": load, "rate_req_s": load * sat,
                      "achieved_arrival_req_s": args.requests / wall if wall else None,
                      "max_arrival_lag_s": late, "requests": args.requests,
                      "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                      "mean_ms": st["mean_ms"], "req_per_s": st["req_per_s"],
                      "eigs_per_s": st["eigs_per_s"], "mean_inflight": st["mean_inflight"],
                      "peak_mem_gb": st["peak_mem_bytes"] / 1e9, "failed": st["failed"],
                      "wall_s": wall, "clocks": clk})
    if rank == 0:
        head = loads[-1] if loads else None
        line = {"metric": "serve p50/p99 latency and throughput",
                "value": head["eigs_per_s"] if head else st_b["eigs_per_s"], "unit": "eigs/s",
                "n_gpus": 1, "steps": len(loads), "warmup": 0,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "serve", "n": "log-uniform [64, 8192]",
                           "select": wl["select"], "q": wl["q"], "precision": args.precision,
                           "mem_cap_gb": wl["mem_cap"] / 1e9,
                           "requests_per_load": args.requests,
                           "forms": "independent, from the seeded generator, made by "
                                    f"{workers} host threads ahead of arrival",
                           "arrivals": "Poisson at load x saturated req/s"},
                "clocks": head["clocks"] if head else clk_b,
                "serve": {"saturated": {"requests": burst, "req_per_s": sat,
                                        "eigs_per_s": st_b["eigs_per_s"],
                                        "p50_ms": st_b["p50_ms"], "p99_ms": st_b["p99_ms"],
                                        "mean_inflight": st_b["mean_inflight"],
                                        "wall_s": wall_b, "clocks": clk_b},
                          "loads": loads}}
        print(json.dumps(line), flush=True)
    return 0


def eigvec_cpu_sample(S, Q, step=16):
    """The eigenvector oracle on every step-th eigenvalue of the form: the
    back substitution (plain C, one core) and the back-transformation (one
    numpy matrix product, BLAS threads) timed separately and scaled to all
    eigenvectors by their work (sum of (j + nb)^2 for the back substitution,
    columns for the back-transformation)."""
    import oracle
    n = S.shape[0]
    pos, j = [], 0
    while j < n:
        nb = 2 if (j + 1 < n and S[j + 1, j] != 0) else 1
        pos.append((j, nb))
        j += nb
    chosen = pos[::step]
    sel = np.zeros(n, dtype=np.int32)
    for j, nb in chosen:
        sel[j] = 1
    t0 = time.perf_counter()
    Y, kinds, _, _ = oracle.eigenvectors(S, None, sel)
    t1 = time.perf_counter()
    X = oracle.normalize_columns(Q @ Y, kinds)
    t2 = time.perf_counter()
    work = sum((j + nb) ** 2 * nb for j, nb in chosen)
    full = sum((j + nb) ** 2 * nb for j, nb in pos)
    est = (t1 - t0) * full / work + (t2 - t1) * n / X.shape[1]
    cores = len(os.sched_getaffinity(0))
    return {"value": n / est, "unit": "eigenvectors/s", "cores": cores, "kind": "oracle",
            "secs": t2 - t0,
            "sample": (f"{X.shape[1]} of {n} eigenvectors (every {step}th eigenvalue): back "
                       f"substitution {t1 - t0:.2f} s on 1 core, back-transformation "
                       f"{t2 - t1:.2f} s (numpy/BLAS, up to {cores} threads); scaled by work "
                       f"to all eigenvectors (est. {est:.1f} s)")}


def run_gen(args, wl):
    """Generalized reordering of the n = 4000 pair (S, T) with Q and Z
    (Eq. 7, second form): selected eigenvalues reordered per second."""
    import torch
    import paper_1905_04975_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()
    mats = si.gen_config(wl["name"])
    sel = mats[4]
    S_np = mats[0]
    n = S_np.shape[0]
    nsel = expected_selected(S_np, sel)
    pristine = [g.to_device(X) for X in mats[:4]]
    work = [g.to_device(X) for X in mats[:4]]
    stream = torch.cuda.Stream()
    opts = g.make_opts(window=wl["window"], chain=wl["chain"], timing=True, sched=args.sched,
                       precision=args.precision)

    def step():
        with torch.cuda.stream(stream):
            for a, b in zip(work, pristine):
                a.copy_(b)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = g.reorder_gen(*work, sel, opts=opts, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        r, _ = step()
        assert r.status == 0, r.status
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            r, t = step()
            ms.append(t)
            stats.append(r.stats)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    value, total_ms = whole_job_rate(nsel * args.steps, sum(ms), dist, "cuda")
    st0 = stats[0]
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)
    flops_iss = st0.upd_flops_issued if st0.upd_flops_issued > 0 else st0.upd_flops
    if args.sched == "persistent" and args.precision == "ozaki":
        ms_k = sum(s.ms_sched for s in stats) / len(stats)
        bf16_peak = pk["bf16_tflops"]
        work = 28.0 * st0.upd_flops + st0.win_flops * (bf16_peak / fp64_peak)
        achieved = work / (ms_k / 1e3) / 1e12
        roof = {"kernel": "sched_kernel<pair> (persistent: pair window tasks + bf16 slice-product "
                          "tiles of S, T, Q, Z)",
                "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak, "traffic": NCU_TRAFFIC.get((wl["name"], "ozaki")),
                "peak_source": f"{src} bf16 {bf16_peak} TF/s",
                "flops_per_launch": work, "bf16_slice_flops": 28.0 * st0.upd_flops,
                "fp64_window_flops": st0.win_flops, "avg_launch_ms": ms_k,
                "critical_path_model_ms": sum(s.sched_cp_ms for s in stats) / len(stats),
                "share_of_step": ms_k / (total_ms / args.steps),
                "note": "latency-bound: the pair window tasks on the critical path set the time"}
        kern = None
    elif args.sched == "persistent":
        ms_k = sum(s.ms_sched for s in stats) / len(stats)
        kern = (f"sched_kernel<pair> (persistent: pair window tasks + "
                f"{fp64_roof_basis(args.precision, pk, src)[0]} of S, T, Q, Z)")
        work_fl = flops_iss + st0.win_flops
    else:
        ms_k = sum(s.ms_update for s in stats) / len(stats)
        kern = (f"update_gen_kernel ({fp64_roof_basis(args.precision, pk, src)[0]}: "
                "Y <- Y U on S, T, Q, Z)")
        work_fl = flops_iss
    if kern is not None:
        achieved = work_fl / (ms_k / 1e3) / 1e12
        _, bound, fpk, fsrc = fp64_roof_basis(args.precision, pk, src)
        roof = {"kernel": kern, "bound": bound, "achieved": achieved, "peak": fpk,
                "unit": "TFLOP/s", "frac": achieved / fpk,
                "traffic": NCU_TRAFFIC.get((wl["name"], args.sched + "-" + args.precision)),
                "peak_source": fsrc,
                "flops_per_launch": work_fl, "update_flops_dense": st0.upd_flops,
                "update_flops_issued": flops_iss, "window_flops": st0.win_flops,
                "avg_launch_ms": ms_k,
                "critical_path_model_ms": sum(s.sched_cp_ms for s in stats) / len(stats),
                "share_of_step": ms_k / (total_ms / args.steps)}
    e2e = None
    if args.e2e_steps > 0:
        pins = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in range(4)]
        views = [p.numpy().T for p in pins]  # Fortran-ordered views of the pinned buffers
        et = []
        for i in range(args.e2e_steps + 1):
            for v, X in zip(views, mats[:4]):
                v[:] = X
            t0 = time.perf_counter()
            g.reorder_gen_host(*views, sel, opts=opts, stream=stream)
            dt = time.perf_counter() - t0
            if i > 0:
                et.append(dt)
        e2e = {"value": nsel * len(et) / sum(et) * world, "unit": "eigs/s",
               "h2d_bytes_per_step": 4 * n * n * 8 + 4 * n,
               "d2h_bytes_per_step": 4 * n * n * 8 + 2 * 8 * n}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cpu = cpu_oracle_sample(S_np, mats[2], sel, what="pair workload",
                                run=lambda ss: oracle.gen_reorder(*mats[:4], ss))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "eigs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "select": wl["select"],
                           "selected_eigs": nsel, "q": wl["q"], "window": wl["window"],
                           "chain": wl["chain"], "precision": args.precision,
                           "sched": args.sched,
                           "l2": "S, T, Q, Z (512 MB > L2) restored from device copies before "
                                 "each step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": int(sum(s.launches for s in stats)),
                "detail": {"windows": int(st0.windows), "chains": int(st0.chains),
                           "tasks": int(st0.tasks), "swaps": int(st0.swaps),
                           "ms_graph": st0.ms_graph, "ms_order": st0.ms_order}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def sweep_cpu(H, Q, sh):
    """The sweep oracle on the whole workload (a few seconds on one core)."""
    import oracle
    t0 = time.perf_counter()
    st, _, _ = oracle.qr_sweep(H, Q, sh)
    dt = time.perf_counter() - t0
    assert st == 0
    return {"value": len(sh) / dt, "unit": "shifts/s", "cores": 1, "kind": "oracle", "secs": dt,
            "sample": f"the whole n={H.shape[0]} sweep with {len(sh)} shifts, {dt:.1f} s on 1 core"}


def run_sweep(args, wl):
    """One bulge-chasing sweep (Section 3.2) on the n = 4000 Hessenberg
    matrix with 64 shifts: shifts chased per second."""
    import torch
    import paper_1905_04975_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()
    H_np, Q_np, sh = si.sweep_config(wl["name"])
    n = H_np.shape[0]
    H0, Q0 = g.to_device(H_np), g.to_device(Q_np)
    H, Q = g.to_device(H_np), g.to_device(Q_np)
    stream = torch.cuda.Stream()
    opts = g.make_opts(window=wl["window"], chain=wl["chain"], timing=True, sched=args.sched)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device="cuda")  # > L2

    def step():
        with torch.cuda.stream(stream):
            H.copy_(H0)
            Q.copy_(Q0)
            flush.fill_(1.0)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = g.qr_sweep(H, Q, sh, opts=opts, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            r, t = step()
            ms.append(t)
            stats.append(r.stats)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    nsh = len(sh)
    value, total_ms = whole_job_rate(nsh * args.steps, sum(ms), dist, "cuda")
    st0 = stats[0]
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)
    flops_iss = st0.upd_flops_issued if st0.upd_flops_issued > 0 else st0.upd_flops
    if args.sched == "persistent":
        ms_k = sum(s.ms_sched for s in stats) / len(stats)
        kern = (f"sched_kernel<sweep> (persistent: bulge-chasing window tasks + "
                f"{fp64_roof_basis(args.precision, pk, src)[0]})")
        work_fl = flops_iss + st0.win_flops
    else:
        ms_k = sum(s.ms_update for s in stats) / len(stats)
        kern = f"update_kernel ({fp64_roof_basis(args.precision, pk, src)[0]}: Y <- Y U)"
        work_fl = flops_iss
    achieved = work_fl / (ms_k / 1e3) / 1e12
    _, bound, fpk, fsrc = fp64_roof_basis(args.precision, pk, src)
    roof = {"kernel": kern, "bound": bound, "achieved": achieved, "peak": fpk,
            "unit": "TFLOP/s", "frac": achieved / fpk,
            "traffic": NCU_TRAFFIC.get((wl["name"], args.sched + "-" + args.precision)),
            "peak_source": fsrc,
            "flops_per_launch": work_fl, "update_flops_dense": st0.upd_flops,
            "update_flops_issued": flops_iss, "window_flops": st0.win_flops,
            "avg_launch_ms": ms_k,
            "critical_path_model_ms": sum(s.sched_cp_ms for s in stats) / len(stats),
            "share_of_step": ms_k / (total_ms / args.steps)}
    e2e = None
    if args.e2e_steps > 0:
        hH = torch.from_numpy(np.asfortranarray(H_np).T.copy()).pin_memory()
        hQ = torch.from_numpy(np.asfortranarray(Q_np).T.copy()).pin_memory()
        oH = torch.empty((n, n), dtype=torch.float64).pin_memory()
        oQ = torch.empty((n, n), dtype=torch.float64).pin_memory()
        et = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                H.t().copy_(hH, non_blocking=True)
                Q.t().copy_(hQ, non_blocking=True)
            g.qr_sweep(H, Q, sh, opts=opts, stream=stream)
            with torch.cuda.stream(stream):
                oH.copy_(H.t(), non_blocking=True)
                oQ.copy_(Q.t(), non_blocking=True)
            stream.synchronize()
            if i > 0:
                et.append(time.perf_counter() - t0)
        e2e = {"value": nsh * len(et) / sum(et) * world, "unit": "shifts/s",
               "h2d_bytes_per_step": 2 * n * n * 8 + 16 * nsh,
               "d2h_bytes_per_step": 2 * n * n * 8}
    cpu = sweep_cpu(H_np, Q_np, sh) if (rank == 0 and not args.no_cpu_baseline) else None
    if rank == 0:
        line = {"metric": SWEEP_METRIC, "value": value, "unit": "shifts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "shifts": nsh, "q": wl["q"],
                           "window": wl["window"], "chain": wl["chain"], "sched": args.sched,
                           "l2": "H, Q restored and a 256 MB buffer written before each step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": int(sum(s.launches for s in stats)),
                "detail": {"windows": int(st0.windows), "chains": int(st0.chains),
                           "tasks": int(st0.tasks), "ms_graph": st0.ms_graph,
                           "ms_order": st0.ms_order}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_eigvec(args, wl):
    """Eigenvectors (Eq. 5) of every eigenvalue of the n = 4000 Schur form,
    back-transformed by its Q (Eq. 6): eigenvectors per second."""
    import torch
    import paper_1905_04975_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()
    S_np, Q_np, _ = make_inputs(wl)
    n = S_np.shape[0]
    S, Q = g.to_device(S_np), g.to_device(Q_np)
    X = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device="cuda")  # > L2

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st = g.GbrEvStats()
        e0.record(stream)
        g.eigenvectors(S, Q, None, stream=stream, stats=st, out=X)
        e1.record(stream)
        e1.synchronize()
        return st, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, sts = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            st, t = step()
            ms.append(t)
            sts.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    value, total_ms = whole_job_rate(n * args.steps, sum(ms), dist, "cuda")
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)
    ms_s = sum(s.ms_solve for s in sts) / len(sts)
    ms_b = sum(s.ms_backtransform for s in sts) / len(sts)
    f_s, f_b = sts[0].solve_flops, sts[0].backtransform_flops
    if ms_b >= ms_s:
        roof = {"kernel": "evgemm_kernel (X = Q Y, DMMA)", "bound": "tensor",
                "achieved": f_b / (ms_b / 1e3) / 1e12, "unit": "TFLOP/s",
                "flops_per_launch": f_b, "avg_launch_ms": ms_b,
                "traffic": NCU_TRAFFIC.get((wl["name"], "evgemm"))}
    else:
        roof = {"kernel": "eigvec_kernel (back substitution, FP64 FMA)", "bound": "alu",
                "achieved": f_s / (ms_s / 1e3) / 1e12, "unit": "TFLOP/s",
                "flops_per_launch": f_s, "avg_launch_ms": ms_s}
    roof.setdefault("traffic", None)
    roof.update({"peak": fp64_peak, "frac": roof["achieved"] / fp64_peak,
                 "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 "
                                 "1.25/2250"),
                 "share_of_step": roof["avg_launch_ms"] / (total_ms / args.steps),
                 "other": {"solve_ms": ms_s, "solve_tflops": f_s / (ms_s / 1e3) / 1e12,
                           "backtransform_ms": ms_b,
                           "backtransform_tflops": f_b / max(ms_b, 1e-9) / 1e9}})
    # end to end: S, Q from pinned host memory, X back, every step
    e2e = None
    if args.e2e_steps > 0:
        hS = torch.from_numpy(np.asfortranarray(S_np).T.copy()).pin_memory()
        hQ = torch.from_numpy(np.asfortranarray(Q_np).T.copy()).pin_memory()
        hX = torch.empty((n, n), dtype=torch.float64).pin_memory()
        et = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                S.t().copy_(hS, non_blocking=True)
                Q.t().copy_(hQ, non_blocking=True)
            g.eigenvectors(S, Q, None, stream=stream, out=X)
            with torch.cuda.stream(stream):
                hX.copy_(X.t(), non_blocking=True)
            stream.synchronize()
            if i > 0:
                et.append(time.perf_counter() - t0)
        e2e = {"value": n * len(et) / sum(et) * world, "unit": "eigenvectors/s",
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = eigvec_cpu_sample(S_np, Q_np)
    if rank == 0:
        line = {"metric": "eigenvectors computed per second", "value": value,
                "unit": "eigenvectors/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "eigenvectors": f"all ({n})",
                           "q": wl["q"], "l2": "256 MB buffer written before each step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": 4 * args.steps}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def measure_reorder(args, g, torch, dist, wl, prec, S_np, Q_np, sel, S, Q, S0, Q0, stream,
                    nsel, local, with_error):
    """Warm-up, timed steps (CUDA events on the library's stream, clocks
    sampled), the dominant kernel's roofline, the end-to-end rate through
    gbr_reorder_host and the accuracy of one more reordering, for one
    precision of the off-diagonal updates."""
    n = S_np.shape[0]
    opts = g.make_opts(window=wl["window"], chain=wl["chain"], precision=prec, timing=True,
                       sched=args.sched)

    def step():
        with torch.cuda.stream(stream):
            S.copy_(S0)
            Q.copy_(Q0)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = g.reorder(S, Q, sel, opts=opts, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        r, _ = step()
        assert r.status == 0, r.status
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            r, t = step()
            ms.append(t)
            stats.append(r.stats)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    value, total_ms = whole_job_rate(nsel * args.steps, sum(ms), dist, "cuda")

    # dominant kernel and its roofline.  With the persistent scheduler one
    # kernel runs every window task and update tile; a large pass runs as
    # three consecutive launches of it (the host orders the later chunks'
    # task graphs while the earlier ones run).  The other launches of a step
    # are the validation, block-scan and eigenvalue kernels (no swap of these
    # workloads is rejected, so there is no re-planning scan).
    st0 = stats[0]
    nsched = max(1, int(st0.launches) - 3)
    nwin = st0.windows
    flops_upd = st0.upd_flops
    flops_win = st0.win_flops
    flops_iss = st0.upd_flops_issued if st0.upd_flops_issued > 0 else flops_upd
    ms_sched = sum(s.ms_sched for s in stats) / len(stats)
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)   # bf16 measured x nominal FP64/bf16
    cp_ms = sum(s.sched_cp_ms for s in stats) / len(stats)
    if ms_sched > 0 and prec == "ozaki":
        # Split-precision updates: 28 bf16 slice products per FP64 product on
        # the tensor pipe (the tiles run K = w densely); the window tasks stay
        # FP64.  frac counts the slice products only; frac_min_time adds the
        # time the FP64 window flops need at the FP64 peak.
        bf16_peak = pk["bf16_tflops"]
        slice_flops = 28.0 * flops_upd
        achieved = slice_flops / (ms_sched / 1e3) / 1e12
        min_s = slice_flops / (bf16_peak * 1e12) + flops_win / (fp64_peak * 1e12)
        roof = {"kernel": "sched_kernel (persistent: FP64 window tasks + bf16 slice-product "
                          "update tiles)",
                "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak,
                "traffic": NCU_TRAFFIC.get((wl["name"], "ozaki")),
                "peak_source": f"{src} bf16 {bf16_peak} TF/s",
                "flops_per_launch": slice_flops / nsched, "bf16_slice_flops": slice_flops,
                "fp64_window_flops": flops_win, "launches_per_step": nsched,
                "frac_min_time": min_s / (ms_sched / 1e3),
                "avg_launch_ms": ms_sched / nsched, "kernel_ms_per_step": ms_sched,
                "critical_path_model_ms": cp_ms,
                "share_of_step": ms_sched / (total_ms / args.steps)}
    elif ms_sched > 0 and prec == "fma":
        # FP64 on the FMA pipe: flops the tiles issued (all-zero rows of U
        # skipped) plus the in-window FP64 flops of accepted swaps, against
        # the FP64 FMA rate from the unit counts and the clock
        achieved = (flops_iss + flops_win) / (ms_sched / 1e3) / 1e12
        alu_peak = FP64_FMA_PEAK
        roof = {"kernel": "sched_kernel (persistent: window tasks + FP64 FMA update tiles)",
                "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": NCU_TRAFFIC.get((wl["name"], "fma")),
                "peak_source": FP64_FMA_PEAK_SOURCE,
                "frac_of_fp64_tensor_peak": achieved / fp64_peak,
                "flops_per_launch": (flops_iss + flops_win) / nsched, "launches_per_step": nsched,
                "update_flops_dense": flops_upd, "update_flops_issued": flops_iss,
                "critical_path_model_ms": cp_ms,
                "avg_launch_ms": ms_sched / nsched, "kernel_ms_per_step": ms_sched,
                "share_of_step": ms_sched / (total_ms / args.steps)}
    elif ms_sched > 0:
        # flops the DMMA tiles issued (the all-zero rows of U are skipped)
        # plus the in-window FP64 flops of accepted swaps
        achieved = (flops_iss + flops_win) / (ms_sched / 1e3) / 1e12
        roof = {"kernel": "sched_kernel (persistent: window tasks + DMMA update tiles)",
                "bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": NCU_TRAFFIC.get((wl["name"], "dmma")),
                "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 "
                                "1.25/2250 (FP64 DMMA probe: 1.047 TF/s)"),
                "flops_per_launch": (flops_iss + flops_win) / nsched, "launches_per_step": nsched,
                "update_flops_dense": flops_upd, "update_flops_issued": flops_iss,
                "critical_path_model_ms": cp_ms,
                "avg_launch_ms": ms_sched / nsched, "kernel_ms_per_step": ms_sched,
                "share_of_step": ms_sched / (total_ms / args.steps)}
    else:
        ms_upd = sum(s.ms_update for s in stats) / len(stats)
        ms_win = sum(s.ms_window for s in stats) / len(stats)
        achieved = flops_iss / (ms_upd / 1e3) / 1e12 if ms_upd > 0 else None
        tname, bound, fpk, _ = fp64_roof_basis(prec, pk, src)
        roof = {"kernel": f"update_kernel ({tname}: Y <- Y U)", "bound": bound,
                "achieved": achieved, "peak": fpk, "unit": "TFLOP/s",
                "frac": achieved / fpk if achieved else None, "traffic": None,
                "launches_per_step": nwin, "avg_launch_ms": ms_upd / max(nwin, 1),
                "share_of_step": ms_upd / (total_ms / args.steps), "window_ms": ms_win}

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if args.e2e_steps > 0:
        Sp = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Qp = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Sh = Sp.numpy().T  # Fortran-ordered view of the pinned buffer
        Qh = Qp.numpy().T
        et, ek, ec, el = [], [], [], []
        with ClockSampler(local) as eclk:
            for i in range(args.e2e_steps + 1):
                Sh[:] = S_np
                Qh[:] = Q_np
                t0 = time.perf_counter()
                r = g.reorder_host(Sh, Qh, sel, opts=opts, stream=stream)
                dt = time.perf_counter() - t0
                assert r.status == 0, r.status
                if i > 0:
                    et.append(dt)
                    ek.append(r.stats.ms_sched if r.stats.ms_sched > 0
                              else r.stats.ms_window + r.stats.ms_update)
                    ec.append(r.stats.ms_h2d + r.stats.ms_d2h)
                    el.append(r.stats.ms_total)
        world = dist.get_world_size() if dist else 1
        e2e = {"value": nsel * len(et) / sum(et) * world, "unit": "eigs/s",
               "steps": len(et), "ms_per_step": 1e3 * sum(et) / len(et),
               "step_ms": [round(1e3 * x, 2) for x in et],
               "kernel_ms": [round(x, 2) for x in ek], "copy_ms": [round(x, 2) for x in ec],
               "library_ms": [round(x, 2) for x in el], "clocks": eclk.summary(),
               "h2d_bytes_per_step": 2 * n * n * 8 + 4 * n,
               "d2h_bytes_per_step": 2 * n * n * 8 + 2 * 8 * n}
        del Sp, Qp
    err = None
    if with_error:
        err = error_report(g, torch, S_np, Q_np, sel, S, Q, S0, Q0, opts, stream,
                           with_oracle=args.error)
    return {"value": value, "ms": total_ms / args.steps, "roofline": roof, "e2e": e2e,
            "clocks": clk.summary(), "error": err,
            "gpu_launches": int(sum(s.launches for s in stats)),
            "stats": st0, "fp64_tflops_of_step": (flops_iss + flops_win)
            / (total_ms / args.steps / 1e3) / 1e12}


def run_reorder(args, wl):
    """One reordering per step on the device-resident workload; for the
    clustered n = 16000 workload both precisions of the off-diagonal updates
    (FP64 DMMA in the line's own fields, split precision in its
    `split_precision` record) with the accuracy of each result."""
    import torch
    import paper_1905_04975_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()

    S_np, Q_np, sel = make_inputs(wl)
    n = S_np.shape[0]
    nsel = expected_selected(S_np, sel)
    S0, Q0 = g.to_device(S_np), g.to_device(Q_np)
    S, Q = g.to_device(S_np), g.to_device(Q_np)
    stream = torch.cuda.Stream()
    precs = ["fma", "ozaki", "dmma"] if args.precision == "both" else [args.precision]
    with_error = args.error or (wl["name"] == "n16000c" and not args.no_error)
    res = {}
    for i, p in enumerate(precs):
        a = args
        if i == 2:
            # the FP64 tensor-core (DMMA) form: a shorter run beside the line
            a = argparse.Namespace(**vars(args))
            a.steps, a.warmup = min(args.steps, args.dmma_steps), min(args.warmup, 1)
            a.e2e_steps = 0
        res[p] = measure_reorder(a, g, torch, dist, wl, p, S_np, Q_np, sel, S, Q, S0, Q0, stream,
                                 nsel, local, with_error and i < 2)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_leg(wl)
    if rank == 0:
        m = res[precs[0]]
        st0 = m["stats"]
        line = {"metric": METRIC, "value": m["value"], "unit": "eigs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": m["ms"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "select": wl["select"],
                           "selected_eigs": nsel, "q": wl["q"], "window": wl["window"],
                           "chain": wl["chain"], "precision": precs[0],
                           "clusters": wl.get("clusters"), "sched": args.sched,
                           "l2": (f"S,Q ({2 * n * n * 8 / 1e9:.2f} GB > L2) restored from a "
                                  "device copy before each step"),
                           "parallelism": f"replicas x{world}"},
                "roofline": m["roofline"], "e2e": m["e2e"], "cpu_baseline": cpu,
                "clocks": m["clocks"], "error": m["error"],
                "gpu_launches": m["gpu_launches"],
                "detail": {"windows": int(st0.windows), "chains": int(st0.chains),
                           "tasks": int(st0.tasks), "swaps": int(st0.swaps),
                           "rejected": int(st0.rejected),
                           "upd_flops": st0.upd_flops, "upd_flops_issued": st0.upd_flops_issued,
                           "win_flops": st0.win_flops,
                           "fp64_tflops_of_step": m["fp64_tflops_of_step"],
                           "host_graph_ms": st0.ms_graph, "host_order_ms": st0.ms_order,
                           # unblocked scalar floor: 12 n flops per adjacent swap (a
                           # rotation on two rows and two columns of S and two of Q)
                           "f_min_flops": f_min_flops(n, int(st0.swaps)),
                           "f_min_tflops_of_step": f_min_flops(n, int(st0.swaps))
                           / (m["ms"] / 1e3) / 1e12}}
        if len(precs) > 1:
            o = res[precs[1]]
            line["split_precision"] = {
                "precision": precs[1], "value": o["value"], "unit": "eigs/s",
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": o["ms"],
                "roofline": o["roofline"], "e2e": o["e2e"], "clocks": o["clocks"],
                "error": o["error"], "gpu_launches": o["gpu_launches"],
                "rejected": int(o["stats"].rejected)}
            line["gpu_launches"] = m["gpu_launches"] + o["gpu_launches"]
        if len(precs) > 2:
            d = res[precs[2]]
            line["fp64_tensor_core"] = {
                "precision": precs[2], "value": d["value"], "unit": "eigs/s",
                "steps": min(args.steps, args.dmma_steps), "warmup": min(args.warmup, 1),
                "ms_per_step": d["ms"], "roofline": d["roofline"], "clocks": d["clocks"],
                "gpu_launches": d["gpu_launches"]}
            line["gpu_launches"] += d["gpu_launches"]
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbr", choices=["gbr", "reference"])
    ap.add_argument("--workload", default="n16000c", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sched", default="persistent", choices=["persistent", "sequential"])
    ap.add_argument("--precision", default=None, choices=["fma", "dmma", "ozaki", "both"],
                    help="off-diagonal updates: FP64 on the FMA pipe, FP64 on the tensor "
                         "cores (DMMA) or split precision (default: both = all three for "
                         "n16000c, else fma)")
    ap.add_argument("--dmma-steps", type=int, default=3,
                    help="both: timed steps of the DMMA form beside the line")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests per load")
    ap.add_argument("--error", action="store_true",
                    help="report the accuracy of one reordering (and vs the oracle, n <= 4000)")
    ap.add_argument("--no-error", action="store_true",
                    help="n16000c: skip the accuracy report")
    ap.add_argument("--loads", type=lambda v: [float(x) for x in v.split(",")],
                    default=[0.7, 0.95], help="serve: arrival rates as fractions of saturation")
    ap.add_argument("--window", type=int, default=None,
                    help="single-reordering workloads: window size w (4..256)")
    ap.add_argument("--chain", type=int, default=None,
                    help="with --window: chain length m (default w / 2)")
    ap.add_argument("--cpu-leg", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.window is not None and wl.get("kind") is None:
        wl["window"] = args.window
        wl["chain"] = args.chain if args.chain is not None else args.window // 2
        if args.window > 128 and args.precision in (None, "both"):
            args.precision = "fma"   # wider windows: FP64 updates only
    if args.cpu_leg:
        return cpu_leg(wl)
    if args.precision is None:
        args.precision = "both" if wl["name"] == "n16000c" else "fma"
    if args.impl == "reference":
        return run_reference(args, wl)
    if wl.get("kind") is not None and args.precision == "both":
        args.precision = "fma"
    if wl.get("kind") == "batch":
        return run_batch(args, wl)
    if wl.get("kind") == "serve":
        return run_serve(args, wl)
    if wl.get("kind") == "eigvec":
        return run_eigvec(args, wl)
    if wl.get("kind") == "gen":
        return run_gen(args, wl)
    if wl.get("kind") == "sweep":
        return run_sweep(args, wl)
    return run_reorder(args, wl)


if __name__ == "__main__":
    sys.exit(main())
