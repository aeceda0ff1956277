"""Multi-GPU runs are replicas (one reordering does not shard without an
exchange per window): every rank runs the same workload, and the job's
rate is all ranks' selected eigenvalues over the slowest rank's time.  This
checks that aggregation with two gloo ranks on the CPU (no GPU)."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "ran" 100 units in 10 (r + 1) ms
        rate, job_ms = bench.whole_job_rate(100, 10.0 * (rank + 1), dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rate": rate, "job_ms": job_ms}, f)


def test_whole_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["job_ms"] == pytest.approx(20.0)           # the slowest rank
        assert r["rate"] == pytest.approx(200 / 0.020)      # both ranks' units


def test_whole_job_rate_single_process():
    import bench
    rate, job_ms = bench.whole_job_rate(50, 25.0)
    assert job_ms == 25.0 and rate == pytest.approx(2000.0)
