"""The multi-rank logic of bench.py on CPU: two gloo ranks (replicas) agree
on the slowest rank's time, the barrier holds, and only rank 0 reports."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # each replica reports its own elapsed time; the job takes the slowest
    out[rank] = bench.max_over_ranks(1.5 + rank, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_max_time():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as manager:
        out = manager.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_algorithmic_bytes_of_the_paper_workload():
    import bench
    w = bench.WORKLOADS["paper"]
    assert bench.algorithmic_bytes(w) == 27_782_400_000
    assert bench.pull_bytes(w) == 27_585_600_000
