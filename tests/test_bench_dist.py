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


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """`bench.py --impl reference` on the host cores: one JSON line with the
    keys of the benchmark contract (sample kept tiny here)."""
    import argparse
    import json
    import bench
    monkeypatch.setattr(bench, "REFERENCE_SECONDS", 1e-3)
    args = argparse.Namespace(steps=2, warmup=1, gpus=1, workload="paper")
    bench.run_reference(args, bench.WORKLOADS["paper"], 1, 0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "edges/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 1)
    assert line["ms_per_step"] > 0 and line["data"] == "synthetic"
    assert line["config"]["name"] == "paper" and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "R-MAT scale 14" in cb["sample"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["machine"]
    assert line["e2e"] == {"value": line["value"], "unit": "edges/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks(capsys):
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, workload="paper")
    bench.run_reference(args, bench.WORKLOADS["paper"], 2, 1)
    assert capsys.readouterr().out == ""


def test_ncu_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The committed DRAM figure is reported only while the profile's source
    digest matches the current edge-pass sources; after any change to them
    the bench reports null."""
    import bench
    csrc = tmp_path / "paper_2402_04403_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gee_csr.cu").write_text("kernel v1\n")
    (csrc / "gee_internal.cuh").write_text("header\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.source_digest()
    (tmp_path / "profiles" / "k_pull_paper.md").write_text(
        f"source_digest: {digest}\ntraffic_bytes_per_launch: 2.862e10\n")
    assert bench.ncu_traffic("k_pull", "paper") == 2.862e10
    assert bench.ncu_traffic("k_pull", "rmat24") is None      # no summary
    (csrc / "gee_csr.cu").write_text("kernel v2\n")
    assert bench.source_digest() != digest
    assert bench.ncu_traffic("k_pull", "paper") is None
