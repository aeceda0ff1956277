#!/usr/bin/env python
"""Benchmark: selected eigenvalues reordered per second on one GB300.

Workload (default): a real Schur form of order n = 4000 from the seeded
generator (60% of positions in 1x1 blocks, 40% in standardized 2x2 blocks,
N(0,1) strict upper part), Q = product of 64 seeded Householder reflectors,
35% of the eigenvalues selected, window 128, chain 64, FP64 DMMA updates.

A step is one full reordering (every planner, window, update and eigenvalue
kernel of the call).  S and Q (256 MB, larger than L2) are restored from a
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
    "n400": dict(name="n400", n=400, select=0.30, q="identity", window=128, chain=64),
    "n16000c": dict(name="n16000c", n=16000, select=0.50, q="64 Householder reflectors",
                    window=128, chain=64),
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
METRIC = "selected eigenvalues reordered per second"

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the current kernels (the sched_kernel captures under profiles/);
# a workload has no entry while no capture of the current build exists.
NCU_TRAFFIC = {("n4000", "dmma"): 1.909980e9 + 2.635823e9,
               ("n4000", "ozaki"): 3.083860e9 + 5.508523e9,
               ("eigvec4000", "evgemm"): 1.052943e9 + 0.125283e9,
               ("g4000", "persistent"): 11.265847e9 + 13.376260e9,
               ("h4000", "persistent"): 0.220709e9 + 0.187885e9,
               ("g4000", "ozaki"): 15.672467e9 + 25.754819e9}


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


def cpu_oracle_sample(S, Q, sel, budget_s=15.0, run=None, what="workload"):
    """Time the oracle on the first k selected blocks (top to bottom) of the
    workload, k grown until ~budget_s of work, and extrapolate to the whole
    workload by the number of adjacent block swaps it needs.  run(sub_sel)
    runs the oracle and returns its result dict (default: the standard-form
    reordering of (S, Q))."""
    import oracle
    if run is None:
        run = lambda sub_sel: oracle.reorder(S, Q, sub_sel)
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

    def swaps_needed(k_blocks):
        cnt, unsel_above, taken = 0, 0, 0
        for b, flag in enumerate(selb):
            if flag:
                if taken >= k_blocks:
                    break
                cnt += unsel_above
                taken += 1
            else:
                unsel_above += 1
        return cnt

    nsel_blocks = sum(selb)
    full_swaps = swaps_needed(nsel_blocks)
    k = max(1, nsel_blocks // 8)
    while True:
        sub_sel = np.zeros(n, np.int32)
        taken = 0
        for s, sz, flag in zip(starts, sizes, selb):
            if flag and taken < k:
                sub_sel[s:s + sz] = 1
                taken += 1
        t0 = time.perf_counter()
        r = run(sub_sel)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or k >= nsel_blocks:
            break
        k = min(nsel_blocks, int(k * 1.6) + 1)
    est_full = dt * full_swaps / max(r["nswaps"], 1)
    nsel = int(np.sum([sz for sz, f in zip(sizes, selb) if f]))
    return {"value": nsel / est_full, "unit": "eigs/s", "cores": 1, "kind": "oracle",
            "sample": (f"first {k} of {nsel_blocks} selected blocks of the n={n} {what} "
                       f"({r['nswaps']} of {full_swaps} block swaps) timed {dt:.1f} s on 1 core, "
                       f"scaled by swap count to the full workload (est. {est_full:.0f} s)")}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if wl.get("kind") == "serve":
        base = si.serve_base(wl["nmax"])
        reqs = si.request_stream(args.requests, seed=1000, nmin=wl["nmin"], nmax=wl["nmax"],
                                 pmin=0.1, pmax=0.6)
        # the oracle's cost grows as n^3: its sample takes the requests of
        # order <= 1024 of the stream, in order
        probs = [si.serve_request(base, n, p, sd) for _, n, p, sd in reqs if n <= 1024][:200]
        nsel = int(sum(expected_selected(S, sel) for S, _, sel in probs))
        sample = lambda: batch_cpu_sample(probs, budget_s=6.0)
        cfg = {"workload": "serve", "n": "requests of order <= 1024 of the stream",
               "select": wl["select"], "q": wl["q"]}
    elif wl.get("kind") == "eigvec":
        S, Q, _ = make_inputs(wl)
        n = S.shape[0]
        times, samples = [], []
        for i in range(args.warmup + args.steps):
            cb = eigvec_cpu_sample(S, Q)
            if i >= args.warmup:
                times.append(n / cb["value"])
                samples.append(cb["sample"])
        value = n * len(times) / sum(times)
        line = {"impl": "reference", "metric": "eigenvectors computed per second", "value": value,
                "unit": "eigenvectors/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "eigenvectors": f"all ({n})",
                           "q": wl["q"]},
                "cpu_baseline": {"value": value, "unit": "eigenvectors/s", "cores": cb["cores"],
                                 "kind": "oracle", "sample": samples[-1]},
                "e2e": {"value": value, "unit": "eigenvectors/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    elif wl.get("kind") == "sweep":
        H, Q, sh = si.sweep_config(wl["name"])
        times, samples = [], []
        for i in range(args.warmup + args.steps):
            cb = sweep_cpu(H, Q, sh)
            if i >= args.warmup:
                times.append(len(sh) / cb["value"])
                samples.append(cb["sample"])
        value = len(sh) * len(times) / sum(times)
        line = {"impl": "reference", "metric": SWEEP_METRIC, "value": value, "unit": "shifts/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": wl["n"], "shifts": wl["shifts"],
                           "q": wl["q"], "window": wl["window"], "chain": wl["chain"]},
                "cpu_baseline": {"value": value, "unit": "shifts/s", "cores": 1, "kind": "oracle",
                                 "sample": samples[-1]},
                "e2e": {"value": value, "unit": "shifts/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    elif wl.get("kind") == "gen":
        import oracle
        S, T, Q, Z, sel = si.gen_config(wl["name"])
        nsel = int(expected_selected(S, sel))
        sample = lambda: cpu_oracle_sample(
            S, Q, sel, budget_s=8.0, what="pair workload",
            run=lambda ss: oracle.gen_reorder(S, T, Q, Z, ss))
        cfg = {"workload": wl["name"], "n": wl["n"], "select": wl["select"], "q": wl["q"],
               "window": wl["window"], "chain": wl["chain"]}
    elif wl.get("kind") == "batch":
        probs = batch_inputs(wl)
        nsel = int(sum(expected_selected(S, sel) for S, _, sel in probs))
        sample = lambda: batch_cpu_sample(probs, budget_s=6.0)
        cfg = {"workload": wl["name"], "instances": wl["count"],
               "n": f"U{{{wl['nmin']}..{wl['nmax']}}}", "select": wl["select"], "q": wl["q"]}
    else:
        S, Q, sel = make_inputs(wl)
        nsel = int(expected_selected(S, sel))
        sample = lambda: cpu_oracle_sample(S, Q, sel, budget_s=8.0)
        cfg = {"workload": wl["name"], "n": wl["n"], "select": wl["select"],
               "q": wl["q"], "window": wl["window"], "chain": wl["chain"]}
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        cb = sample()
        if i >= args.warmup:
            times.append(nsel / cb["value"])
            samples.append(cb["sample"])
    value = nsel * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "eigs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "eigs/s", "cores": 1, "kind": "oracle",
                             "sample": samples[-1]},
            "e2e": {"value": value, "unit": "eigs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
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


def error_report(g, torch, S_np, Q_np, sel, S, Q, S0, Q0, opts, stream):
    """Accuracy of one reordering of the workload (after the timed steps):
    residual ||A - Q S Q^T||_F / ||A||_F and ||Q^T Q - I||_F estimated with 32
    Gaussian probe vectors on the GPU, eigenvalue order against the stable
    partition of the input eigenvalues, and for n <= 4000 the difference to
    the FP64 oracle's result (eigenvalues, leading invariant subspace)."""
    import oracle
    from tests.helpers import block_eigs, expected_order, sin_angle
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
    if n <= 4000:
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


def batch_cpu_sample(probs, budget_s=12.0):
    """The oracle on the first instances of the batch until ~budget_s,
    scaled to the whole batch by selected eigenvalues."""
    import oracle
    t0 = time.perf_counter()
    done = 0
    eigs = 0
    while done < len(probs) and time.perf_counter() - t0 < budget_s:
        S, Q, sel = probs[done]
        oracle.reorder(S, Q, sel)
        eigs += expected_selected(S, sel)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": eigs / dt, "unit": "eigs/s", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(probs)} instances ({eigs} selected eigenvalues) "
                      f"in {dt:.1f} s on 1 core"}


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
    roof = {"kernel": "sched_kernel (persistent, all instances: window tasks + update tiles)",
            "bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": None,
            "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 1.25/2250"),
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


def run_serve(args, wl):
    """Serving: a Poisson stream of requests (n log-uniform, see the
    workload) through the continuous-batching server.  A saturation burst
    first measures the throughput; the stream then arrives at each --load
    fraction of it.  Requests are cut from one base form (schur_inputs)."""
    import torch
    import paper_1905_04975_gb300 as g

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    g.load()
    base = si.serve_base(wl["nmax"], seed=rank)
    reqs = si.request_stream(args.requests, seed=1000 + rank, nmin=wl["nmin"], nmax=wl["nmax"],
                             pmin=0.1, pmax=0.6, rate=1.0)

    def make(i):
        _, n, p, sd = reqs[i % len(reqs)]
        S, Q, sel = si.serve_request(base, n, p, sd)
        nn = S.shape[0]
        # pinned host buffers (the caching host allocator reuses them)
        tS = torch.empty((nn, nn), dtype=torch.float64).pin_memory()
        tQ = torch.empty((nn, nn), dtype=torch.float64).pin_memory()
        hS, hQ = tS.numpy().T, tQ.numpy().T      # Fortran-ordered views
        hS[:] = S
        hQ[:] = Q
        return (tS, tQ, hS, hQ, sel, int(expected_selected(S, sel)))

    def run(rate, count, offset):
        """Submits `count` requests (Poisson arrivals at `rate` per second,
        or all at once when rate is None) and waits for all of them."""
        srv = g.Server(mem_cap_bytes=wl["mem_cap"], precision=args.precision)
        try:
            gaps = np.random.default_rng(7 + offset).exponential(1.0 / rate, count) if rate else None
            pending = {}
            t0 = time.perf_counter()
            t_next = t0
            eigs = 0
            for i in range(count):
                item = make(offset + i)
                if gaps is not None:
                    t_next += gaps[i]
                    dt = t_next - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                t = srv.submit(item[2], item[3], item[4], eigs=False)
                pending[t] = item
                eigs += item[5]
                for tk in [tk for tk in pending if srv.poll(tk) is not None]:
                    del pending[tk]
            for tk in list(pending):
                r = srv.wait(tk, -1)
                assert r.status >= 0, r.status
            wall = time.perf_counter() - t0
            st = srv.stats()
        finally:
            srv.close()
        return st, wall, eigs

    burst = max(20, args.requests // 10)
    st_b, wall_b, eigs_b = run(None, burst, 0)
    sat = st_b["req_per_s"]
    loads = []
    for load in args.loads:
        st, wall, eigs = run(load * sat, args.requests, burst)
        loads.append({"load": load, "rate_req_s": load * sat, "requests": args.requests,
                      "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                      "mean_ms": st["mean_ms"], "req_per_s": st["req_per_s"],
                      "eigs_per_s": st["eigs_per_s"], "mean_inflight": st["mean_inflight"],
                      "peak_mem_gb": st["peak_mem_bytes"] / 1e9, "failed": st["failed"],
                      "wall_s": wall})
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
                           "arrivals": "Poisson at load x saturated req/s"},
                "serve": {"saturated": {"requests": burst, "req_per_s": sat,
                                        "eigs_per_s": st_b["eigs_per_s"],
                                        "p50_ms": st_b["p50_ms"], "p99_ms": st_b["p99_ms"],
                                        "wall_s": wall_b},
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
        kern = "sched_kernel<pair> (persistent: pair window tasks + DMMA tiles of S, T, Q, Z)"
        work_fl = flops_iss + st0.win_flops
    else:
        ms_k = sum(s.ms_update for s in stats) / len(stats)
        kern = "update_gen_kernel (DMMA FP64 Y <- Y U on S, T, Q, Z)"
        work_fl = flops_iss
    if kern is not None:
        achieved = work_fl / (ms_k / 1e3) / 1e12
        roof = {"kernel": kern, "bound": "tensor", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": NCU_TRAFFIC.get((wl["name"], args.sched)),
                "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 "
                                "1.25/2250 (FP64 DMMA probe: 1.047 TF/s)"),
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
    return {"value": len(sh) / dt, "unit": "shifts/s", "cores": 1, "kind": "oracle",
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
        kern = "sched_kernel<sweep> (persistent: bulge-chasing window tasks + DMMA tiles)"
        work_fl = flops_iss + st0.win_flops
    else:
        ms_k = sum(s.ms_update for s in stats) / len(stats)
        kern = "update_kernel (DMMA FP64 Y <- Y U)"
        work_fl = flops_iss
    achieved = work_fl / (ms_k / 1e3) / 1e12
    roof = {"kernel": kern, "bound": "tensor", "achieved": achieved, "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "traffic": NCU_TRAFFIC.get((wl["name"], args.sched)),
            "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 "
                            "1.25/2250 (FP64 DMMA probe: 1.047 TF/s)"),
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbr", choices=["gbr", "reference"])
    ap.add_argument("--workload", default="n4000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sched", default="persistent", choices=["persistent", "sequential"])
    ap.add_argument("--precision", default="dmma", choices=["dmma", "ozaki"])
    ap.add_argument("--requests", type=int, default=400, help="serve: requests per load")
    ap.add_argument("--error", action="store_true",
                    help="report the accuracy of one reordering (and vs the oracle, n <= 4000)")
    ap.add_argument("--loads", type=lambda v: [float(x) for x in v.split(",")],
                    default=[0.5, 0.9], help="serve: arrival rates as fractions of saturation")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
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
    opts = g.make_opts(window=wl["window"], chain=wl["chain"], precision=args.precision,
                       timing=True, sched=args.sched)

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
    # kernel runs every window task and update tile; all of its arithmetic is
    # FP64 (DMMA for the updates, FP64 FMA inside the windows), so its roofline
    # is the FP64 peak and its algorithmic work is the planner's exact update
    # flop count plus the in-window flops the kernel counts.
    st0 = stats[0]
    nwin = st0.windows
    flops_upd = st0.upd_flops
    flops_win = st0.win_flops
    ms_sched = sum(s.ms_sched for s in stats) / len(stats)
    pk, src = peaks()
    fp64_peak = pk["bf16_tflops"] * (1.25 / 2250.0)   # bf16 measured x nominal FP64/bf16
    cp_ms = sum(s.sched_cp_ms for s in stats) / len(stats)
    if ms_sched > 0 and args.precision == "ozaki":
        # Split-precision updates: 28 bf16 slice products per FP64 product,
        # issued on the tensor pipe; the window tasks stay FP64.  The kernel's
        # work in bf16-peak-equivalent flops (window flops scaled by the
        # bf16/FP64 peak ratio), so frac = (minimum time at both peaks) / time.
        bf16_peak = pk["bf16_tflops"]
        work = 28.0 * flops_upd + flops_win * (bf16_peak / fp64_peak)
        achieved = work / (ms_sched / 1e3) / 1e12
        roof = {"kernel": "sched_kernel (persistent: FP64 window tasks + bf16 slice-product "
                          "update tiles)",
                "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak,
                "traffic": NCU_TRAFFIC.get((wl["name"], "ozaki")),
                "peak_source": f"{src} bf16 {bf16_peak} TF/s",
                "flops_per_launch": work, "bf16_slice_flops": 28.0 * flops_upd,
                "fp64_window_flops": flops_win, "launches_per_step": 1,
                "avg_launch_ms": ms_sched, "critical_path_model_ms": cp_ms,
                "share_of_step": ms_sched / (total_ms / args.steps),
                "note": "latency-bound: the window tasks on the critical path set the time"}
    elif ms_sched > 0:
        # flops the DMMA tiles issued: the all-zero rows of U are skipped
        flops_iss = st0.upd_flops_issued if st0.upd_flops_issued > 0 else flops_upd
        achieved = (flops_iss + flops_win) / (ms_sched / 1e3) / 1e12
        roof = {"kernel": "sched_kernel (persistent: window tasks + DMMA update tiles)",
                "bound": "tensor", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": NCU_TRAFFIC.get((wl["name"], "dmma")),
                "peak_source": (f"{src} bf16 {pk['bf16_tflops']} TF/s x nominal FP64/bf16 "
                                "1.25/2250 (FP64 DMMA probe: 1.047 TF/s)"),
                "flops_per_launch": flops_iss + flops_win, "launches_per_step": 1,
                "update_flops_dense": flops_upd, "update_flops_issued": flops_iss,
                "critical_path_model_ms": cp_ms,
                "avg_launch_ms": ms_sched,
                "share_of_step": ms_sched / (total_ms / args.steps)}
    else:
        ms_upd = sum(s.ms_update for s in stats) / len(stats)
        ms_win = sum(s.ms_window for s in stats) / len(stats)
        achieved = flops_upd / (ms_upd / 1e3) / 1e12 if ms_upd > 0 else None
        roof = {"kernel": "update_kernel (DMMA FP64 Y <- Y U)", "bound": "tensor",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak if achieved else None, "traffic": None,
                "launches_per_step": nwin, "avg_launch_ms": ms_upd / max(nwin, 1),
                "share_of_step": ms_upd / (total_ms / args.steps), "window_ms": ms_win}

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if args.e2e_steps > 0:
        Sp = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Qp = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Sh = Sp.numpy().T  # Fortran-ordered view of the pinned buffer
        Qh = Qp.numpy().T
        et = []
        for i in range(args.e2e_steps + 1):
            Sh[:] = S_np
            Qh[:] = Q_np
            t0 = time.perf_counter()
            r = g.reorder_host(Sh, Qh, sel, opts=opts, stream=stream)
            dt = time.perf_counter() - t0
            if i > 0:
                et.append(dt)
        e2e = {"value": nsel * len(et) / sum(et) * world, "unit": "eigs/s",
               "h2d_bytes_per_step": 2 * n * n * 8 + 4 * n,
               "d2h_bytes_per_step": 2 * n * n * 8 + 2 * 8 * n}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(S_np, Q_np, sel)
    err = error_report(g, torch, S_np, Q_np, sel, S, Q, S0, Q0, opts, stream) if args.error else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "eigs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"], "n": n, "select": wl["select"],
                           "selected_eigs": nsel, "q": wl["q"], "window": wl["window"],
                           "chain": wl["chain"], "precision": args.precision, "sched": args.sched,
                           "l2": "S,Q (256 MB > L2) restored from a device copy before each step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
                "clocks": clk.summary(), "error": err,
                "gpu_launches": int(sum(s.launches for s in stats)),
                "detail": {"windows": int(nwin), "chains": int(st0.chains),
                           "tasks": int(st0.tasks), "swaps": int(st0.swaps),
                           "upd_flops": flops_upd, "win_flops": flops_win,
                           "fp64_tflops_of_step": (flops_upd + flops_win)
                           / (total_ms / args.steps / 1e3) / 1e12}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
