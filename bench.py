#!/usr/bin/env python
"""Throughput of the GEE edge-map pass (Z = A W) on GB300.

A step is one full pass of the hot path over one label vector: label check
and class histogram, then the edge pass with the 1/n_k scaling fused in,
writing all of Z -- through the C ABI (gee_embed_graph) on a graph kept
resident as a row-sorted CSR.  The default workload is the paper-scale
synthetic graph: R-MAT (a, b, c) = (0.57, 0.19, 0.19) on 2^26 ids, n =
65,600,000 nodes, s = 1,800,000,000 undirected unit-weight edges, K = 50,
every node labelled.  Inputs (14.4 GB of arcs, 13.1 GB of Z) are far larger
than L2, so no flush is needed between steps.

Printed JSON line (rank 0): value = edges/s over all ranks; `roofline` for
the dominant kernel (k_pull) from CUDA events recorded live on its stream;
`e2e` the same metric through the host-buffer entry point with the label
upload and the Z download inside the timed region; `cpu_baseline` the FP64
oracle on a bounded sample; `oneshot` the edge-list entry point (gee_embed)
that builds nothing resident; `serving` (one GPU) the metric's second half:
1,000 requests of the serving workload through the request loop
(gee_server_*), p50/p99 latency and edges/s beside one-at-a-time plain
calls.

`--impl reference` times the oracle (serial C, FP64) on the host cores
instead, on bounded samples of the same workload.

Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the
data path; a gloo barrier brackets the timed region and the slowest rank's
time is used.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "paper": dict(desc="paper-scale R-MAT (Friendster-sized): n=65.6M, s=1.8B "
                       "undirected unit-weight edges, K=50, all labelled",
                  scale=26, n=65_600_000, s=1_800_000_000, K=50, frac_unlabeled=0.0,
                  weighted=False, laplacian=False, seed=3),
    "paper10": dict(desc="paper-scale R-MAT, 10% of nodes labelled",
                    scale=26, n=65_600_000, s=1_800_000_000, K=50, frac_unlabeled=0.9,
                    weighted=False, laplacian=False, seed=3),
    "rmat24": dict(desc="R-MAT scale 24, edge factor 16, float weights in (0,1], K=20, "
                        "10% unlabelled",
                   scale=24, n=1 << 24, s=268_435_456, K=20, frac_unlabeled=0.1,
                   weighted=True, laplacian=False, seed=2),
    "rmat24multi": dict(desc="R-MAT scale 24 weighted, L=32 label vectors of K=20 in one "
                             "pass (W widened to 640 columns)",
                        scale=24, n=1 << 24, s=268_435_456, K=20, frac_unlabeled=0.1,
                        weighted=True, laplacian=False, seed=2, L=32),
    "batch4096": dict(desc="4,096 independent planted-partition graphs (the edge-sampling "
                           "form of an SBM, p_in/p_out = 10), n log-uniform in [1e3, 1e5], "
                           "average degree uniform in [10, 50], K uniform in {2..32} "
                           "blocks = labels, float weights in (0,1], one batch per step",
                      graphs=4096, n_lo=1e3, n_hi=1e5, deg_lo=10, deg_hi=50, K_lo=2, K_hi=32,
                      ratio=10.0, weighted=True, laplacian=False, seed=4,
                      scale=0, n=0, s=0, K=0),
    "serve": dict(desc="serving: Poisson stream of embedding requests, graphs of 1e3-1e8 edges "
                        "(log-uniform; R-MAT and planted partition half and half; n = s/8), K "
                        "uniform in [2, 64], 30% re-labelings of resident graphs, 80 GiB "
                        "admission budget, host buffers in page-locked memory",
                  pool=64, resident=8, s_lo=1e3, s_hi=1e8, K_lo=2, K_hi=64, relabel=0.3,
                  load=0.8, budget=80 << 30, streams=8, max_batch=256, seed=5,
                  weighted=False, laplacian=False, scale=0, n=0, s=0, K=0),
    "precision": dict(desc="precision ladder: each arithmetic path (uint32 counts, FP32 weight "
                            "sums, FP32 Laplacian, multi-label and batched forms) against the "
                            "FP64 oracle on the tiny SBM (all rows), R-MAT scale 24 and the "
                            "paper-scale graph (sampled rows)",
                      rows=4096, seed=6, weighted=False, laplacian=False,
                      scale=0, n=0, s=0, K=0),
    "unsup": dict(desc="unsupervised GEE: planted partition (edge-sampling SBM, p_in/p_out = "
                        "10), n = 2^24, s = 2^28 unit-weight edges, K = 16 blocks; starting "
                        "labels: the planted block for 10% of nodes, uniform random for the "
                        "rest; rounds of embedding + k-means assignment until nothing moves",
                  n=1 << 24, s=1 << 28, K=16, ratio=10.0, max_iter=40, known=0.1, seed=7,
                  weighted=False, laplacian=False, scale=0),
    "rmat24lap": dict(desc="R-MAT scale 24 weighted, Laplacian variant",
                      scale=24, n=1 << 24, s=268_435_456, K=20, frac_unlabeled=0.1,
                      weighted=True, laplacian=True, seed=2),
}
METRIC = "GEE edges/s and % HBM roofline at 1.8B edges"
PAPER_CONTEXT = ("paper: GEE-Ligra 6.42 s on Friendster (65M nodes, 1.8B edges), "
                 "24-core Xeon 8259CL = 0.28e9 edges/s (different machine and graph)")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest():
    """Digest of the edge-pass kernel sources (the ncu traffic figure is only
    reported while it matches)."""
    h = hashlib.sha256()
    for name in ("gee_csr.cu", "gee_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2402_04403_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    if not m or not d or d.group(1) != source_digest():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.out = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            ident = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            ident = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if ident:
            cmd += ["-i", ident]
        try:
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=self.out, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            text, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            text = ""
        rows = []
        for line in text.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        sm = sorted(r[0] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Random one-byte label gathers that miss L1 cost about one SM clock each in
# the L1 unit: 0.94 per SM clock on any number of SMs and for every load
# form (microbenchmark of random byte loads over a 65.6 MB L2-resident
# array; profiles/k_pull_paper_shift3_full.md).
GATHERS_PER_SM_CLOCK = 0.94


def gather_bound(g, K, prof, clocks):
    """The hub-row kernel's second bound: its label gathers that do not come
    from its shared-memory copy (for K classes), at GATHERS_PER_SM_CLOCK per
    SM clock on every SM, against its measured average launch time."""
    import torch
    if "k_pull_heavy" not in prof:
        return None
    ga = g.gathers(K)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    bound_ms = ga["hub_other"] / (GATHERS_PER_SM_CLOCK * sms * mhz * 1e6) * 1e3
    heavy_ms = prof["k_pull_heavy"]["total_ms"] / max(1, prof["k_pull_heavy"]["launches"])
    return {"kernel": "k_pull_heavy", "bound": "L1 label gathers",
            "gathers_per_launch": ga["hub_other"],
            "shared_memory_labels_per_launch": ga["hub_shared"],
            "rate_per_sm_clock": GATHERS_PER_SM_CLOCK, "sms": sms, "sm_mhz": mhz,
            "bound_ms": bound_ms, "avg_launch_ms": heavy_ms,
            "frac": bound_ms / heavy_ms}


def algorithmic_bytes(w):
    """Compulsory bytes of one step: read the edges (8 B each, +4 B weight),
    read Y once (4 B per node), write Z once (4 B per cell)."""
    return w["s"] * (8 + 4 * w["weighted"]) + 4 * w["n"] + 4 * w["n"] * w["K"]


def pull_bytes(w):
    """Compulsory bytes of the edge-pass kernel: edges, the compact (1 B)
    labels once, Z once."""
    return w["s"] * (8 + 4 * w["weighted"]) + w["n"] + 4 * w["n"] * w["K"]


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def sample_inputs(w, shift, use_gpu):
    """The workload shrunk by 2^shift (same generator, a, b, c, K, label mix)."""
    import numpy as np
    import graphgen
    scale = w["scale"] - shift
    n = max(1, w["n"] >> shift)
    s = max(1, w["s"] >> shift)
    if use_gpu:
        e = graphgen.rmat_edges_device(scale, n, 0, s, w["seed"]).cpu().numpy()
        Y = graphgen.labels_device(n, w["K"], w["seed"] + 1, w["frac_unlabeled"]).cpu().numpy()
        wt = graphgen.weights_device(s, w["seed"] + 2).cpu().numpy() if w["weighted"] else None
    else:
        e = graphgen.rmat_edges(scale, n, 0, s, w["seed"])
        Y = graphgen.labels(n, w["K"], w["seed"] + 1, w["frac_unlabeled"])
        wt = graphgen.weights(s, w["seed"] + 2) if w["weighted"] else None
    return dict(edges=np.ascontiguousarray(e), Y=Y, weights=wt, n=n, s=s, scale=scale)


def time_oracle(sample, w):
    import oracle
    t = time.perf_counter()
    oracle.embed(sample["edges"], sample["Y"], w["K"], weights=sample["weights"],
                 laplacian=w["laplacian"])
    return time.perf_counter() - t


def host_cpu():
    """The host the oracle is timed on: logical CPUs and the CPU model (x86
    'model name', else the Arm implementer/part codes of /proc/cpuinfo)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            fields = dict(l.split(":", 1) for l in fh.read().splitlines() if ":" in l)
        fields = {k.strip(): v.strip() for k, v in fields.items()}
        model = fields.get("model name") or (
            f"implementer {fields['CPU implementer']} part {fields['CPU part']}"
            if "CPU part" in fields else None)
    except (OSError, KeyError, ValueError):
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def cpu_baseline(w, use_gpu, shift=5):
    smp = sample_inputs(w, shift, use_gpu)
    secs = time_oracle(smp, w)
    return {"value": smp["s"] / secs, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": (f"R-MAT scale {smp['scale']}: n={smp['n']}, s={smp['s']} "
                       f"(1/{1 << shift} of the workload, same generator and label mix), "
                       f"serial C FP64 oracle, {secs:.2f} s"),
            "seconds": secs}


# seconds of oracle work one `--impl reference` run aims at
REFERENCE_SECONDS = 120.0


def run_reference(args, w, world, rank):
    if rank != 0:
        return
    import torch
    use_gpu = torch.cuda.is_available()
    # size each step's sample so the whole run stays near REFERENCE_SECONDS
    probe = sample_inputs(w, 12, use_gpu)
    rate = probe["s"] / max(time_oracle(probe, w), 1e-4)
    per_step = REFERENCE_SECONDS / max(1, args.steps + args.warmup)
    shift = 12
    while shift > 4 and (w["s"] >> (shift - 1)) / rate < per_step:
        shift -= 1
    smp = sample_inputs(w, shift, use_gpu)
    for _ in range(args.warmup):
        time_oracle(smp, w)
    times = [time_oracle(smp, w) for _ in range(args.steps)]
    total = sum(times)
    value = smp["s"] * args.steps / total
    sample = (f"R-MAT scale {smp['scale']}: n={smp['n']}, s={smp['s']} per step "
              f"(1/{1 << shift} of the workload), serial C FP64 oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(args, w),
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_for(args, w):
    return {"workload": w["desc"], "name": args.workload, "n": w["n"], "s": w["s"],
            "K": w["K"], "weighted": w["weighted"], "laplacian": w["laplacian"],
            "generator": "R-MAT a=0.57 b=0.19 c=0.19, Philox4x32-10 seed "
                         f"{w['seed']}, ids permuted",
            "graph": "resident row-sorted CSR (built once per graph, ingest timed apart)",
            "l2": "inputs larger than L2, no flush", "parallelism": "replicas",
            "context": PAPER_CONTEXT}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def run_multi(args, w, world, rank, local):
    """L label vectors on one resident graph: one widened pass per step,
    against L single-vector passes on the same graph (same results)."""
    import numpy as np
    import torch

    import graphgen
    import paper_2402_04403_gb300 as gee
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, s, K, L = w["n"], w["s"], w["K"], w["L"]
    edges = graphgen.rmat_edges_device(w["scale"], n, 0, s, w["seed"], device=dev)
    wts = graphgen.weights_device(s, w["seed"] + 2, device=dev) if w["weighted"] else None
    Ys = torch.stack([graphgen.labels_device(n, K, w["seed"] + 100 + l, w["frac_unlabeled"],
                                             device=dev) for l in range(L)])
    g = gee.Graph(edges, n, weights=wts)
    del edges
    Zm = torch.empty((n, L * K), dtype=torch.float32, device=dev)
    Z1 = torch.empty((n, K), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    lap = w["laplacian"]
    for _ in range(args.warmup):
        g.embed_multi(Ys, K, laplacian=lap, out=Zm)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.embed_multi(Ys, K, laplacian=lap, out=Zm)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world) / args.steps
    # per-kernel times of a few more passes (launch tracing, after the timed region)
    gee.profile_read()
    gee.profile_enable(True)
    for _ in range(3):
        g.embed_multi(Ys, K, laplacian=lap, out=Zm)
    torch.cuda.synchronize()
    gee.profile_enable(False)
    kernels = {k: {"launches": v["launches"], "ms": v["total_ms"] / 3}
               for k, v in gee.profile_read().items()}
    # same results in both forms: compare two blocks with single-vector calls
    worst = 0.0
    for l in (0, L - 1):
        g.embed(Ys[l], K, laplacian=lap, out=Z1)
        blk = Zm[:, l * K:(l + 1) * K]
        nz = Z1 != 0
        if nz.any():
            worst = max(worst, ((blk - Z1).abs()[nz] / Z1[nz].abs()).max().item())
    # the plain form: L separate calls, one label vector each
    torch.cuda.synchronize()
    e0.record(stream)
    for l in range(L):
        g.embed(Ys[l], K, laplacian=lap, out=Z1)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    line = {
        "metric": "GEE edge-embeddings/s (L label vectors per pass)", "value": world * L * s / (ms / 1e3),
        "unit": "edge-embeddings/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if (w["weighted"] or lap) else "u32", "data": "synthetic",
        "config": config_for(args, w),
        "plain": {"value": world * L * s / (plain_ms / 1e3), "ms_for_L_calls": plain_ms,
                  "api": "L x gee_embed_graph"},
        "speedup_vs_plain": plain_ms / ms,
        "kernels_per_pass": kernels,
        "max_rel_diff_vs_plain": worst,
    }
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_problems(w, shift=0):
    """Per-graph sizes of the batched workload (seeded): n, average degree,
    K; s = n * degree / 2 edges.  shift shrinks the number of graphs."""
    import numpy as np
    rng = np.random.default_rng(w["seed"])
    G = w["graphs"] >> shift
    n = np.exp(rng.uniform(np.log(w["n_lo"]), np.log(w["n_hi"]), G)).astype(np.int64)
    deg = rng.uniform(w["deg_lo"], w["deg_hi"], G)
    K = rng.integers(w["K_lo"], w["K_hi"] + 1, G)
    s = np.maximum((n * deg / 2).astype(np.int64), 1)
    return n, s, K


def run_batch(args, w, world, rank, local):
    """Many small graphs: one gee_embed_batch per step against one gee_embed
    call per graph (the plain path), same inputs, same results."""
    import ctypes

    import numpy as np
    import torch

    import graphgen
    import paper_2402_04403_gb300 as gee
    from paper_2402_04403_gb300 import _lib
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, s, K = batch_problems(w, args.scale_shift)
    G = len(n)
    e_off = np.concatenate([[0], np.cumsum(s)])
    n_off = np.concatenate([[0], np.cumsum(n)])
    z_off = np.concatenate([[0], np.cumsum(n * K)])
    E = torch.empty((int(e_off[-1]), 2), dtype=torch.int32, device=dev)
    Y = torch.empty(int(n_off[-1]), dtype=torch.int32, device=dev)
    Wt = graphgen.weights_device(int(e_off[-1]), w["seed"] + 1, device=dev)
    Z = torch.empty(int(z_off[-1]), dtype=torch.float32, device=dev)
    Zp = torch.empty_like(Z)
    for g in range(G):
        graphgen.planted_edges_device(int(n[g]), int(K[g]), int(s[g]), w["ratio"],
                                      w["seed"] * 100000 + g, out=E[e_off[g]:e_off[g + 1]])
        graphgen.planted_labels_device(int(n[g]), int(K[g]), out=Y[n_off[g]:n_off[g + 1]])
    torch.cuda.synchronize()
    lib = gee.load()

    def table(out):
        arr = (_lib.Problem * G)()
        for g in range(G):
            arr[g].edges = E[e_off[g]:].data_ptr()
            arr[g].weights = Wt[e_off[g]:].data_ptr()
            arr[g].s = int(s[g])
            arr[g].Y = Y[n_off[g]:].data_ptr()
            arr[g].n = int(n[g])
            arr[g].K = int(K[g])
            arr[g].Z = out[z_off[g]:].data_ptr()
        return arr

    arr = table(Z)
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)
    opts = _lib.options()

    def batch():
        gee.check(lib.gee_embed_batch(arr, G, None, ctypes.byref(opts), sh), "batch")

    plain_args = [(ctypes.c_void_p(arr[g].edges), ctypes.c_void_p(arr[g].weights), arr[g].s,
                   ctypes.c_void_p(arr[g].Y), arr[g].n, arr[g].K,
                   ctypes.c_void_p(Zp[z_off[g]:].data_ptr())) for g in range(G)]

    def plain():
        for a in plain_args:
            gee.check(lib.gee_embed(a[0], a[1], a[2], a[3], a[4], a[5], 0, a[6],
                                    ctypes.byref(opts), sh), "plain")

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world) / steps

    for _ in range(args.warmup):
        batch()
    sampler = ClockSampler(local) if not args.no_clocks else None
    ms = timed(batch, args.steps)
    clocks = sampler.stop() if sampler else None
    gee.profile_read()
    gee.profile_enable(True)
    batch()
    torch.cuda.synchronize()
    gee.profile_enable(False)
    kernels = {k: {"launches": v["launches"], "ms": v["total_ms"]}
               for k, v in gee.profile_read().items()}
    # the plain path with GEE_AUTO tuned on this device (gee_autotune)
    tune_t0 = time.perf_counter()
    table = gee.autotune(0)
    tune_s = time.perf_counter() - tune_t0
    plain()  # warm-up of the plain path
    plain_ms = timed(plain, max(1, min(args.steps, 3)))
    gee.tune_set([])
    # same results: the batch and the plain calls on every graph
    nz = Zp != 0
    worst = ((Z - Zp).abs()[nz] / Zp[nz].abs()).max().item() if nz.any() else 0.0
    zero_ok = bool(torch.all(Z[~nz] == 0).item())
    total_s = int(e_off[-1])
    line = {
        "metric": "GEE edges/s, batch of independent graphs in one launch sequence",
        "value": world * total_s / (ms / 1e3), "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "name": args.workload, "graphs": G,
                   "edges": total_s, "nodes": int(n_off[-1]), "Z_cells": int(z_off[-1]),
                   "api": "gee_embed_batch", "parallelism": "replicas",
                   "l2": "inputs larger than L2, no flush"},
        "plain": {"value": world * total_s / (plain_ms / 1e3), "ms": plain_ms,
                  "api": f"{G} x gee_embed (AUTO strategy, autotuned)",
                  "autotune_seconds": tune_s,
                  "autotune_choices": {k: sum(1 for c in table if c["strategy"] == k)
                                       for k in ("atomic", "private", "segmented")}},
        "speedup_vs_plain": plain_ms / ms,
        "max_rel_diff_vs_plain": worst, "zeros_agree": zero_ok,
        "kernels_per_batch": kernels,
        "gpu_launches": sum(v["launches"] for v in kernels.values()) * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def _host_link_rates(dev, nbytes=1 << 30, reps=3):
    """Copy-engine rates between page-locked host memory and the device
    (GB/s): each direction alone, and both at once on two streams."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_in = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(up, down):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if up:
                with torch.cuda.stream(s1):
                    d_in.copy_(h_in, non_blocking=True)
            if down:
                with torch.cuda.stream(s2):
                    h_out.copy_(d_out, non_blocking=True)
            torch.cuda.synchronize(dev)
            best = min(best, time.perf_counter() - t0)
        return (int(up) + int(down)) * nbytes / best / 1e9

    return {"h2d_gbs": timed(True, False), "d2h_gbs": timed(False, True),
            "both_gbs": timed(True, True), "probe_bytes": nbytes}


def serve_measure(args, w, local, R):
    """Serving (gee_server_*) on R requests: a burst of all requests for the
    server's throughput, then a Poisson stream at `load` x the plain path's
    capacity for its latencies; the plain path is one synchronous host-buffer
    call per request (gee_embed_host, or gee_embed_graph_host on a resident
    graph), whose latencies under the same arrivals follow from its measured
    service times (first-in first-out, one call at a time).  Returns the
    figures as a dict."""
    import threading

    import numpy as np
    import torch

    import graphgen
    import paper_2402_04403_gb300 as gee
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(w["seed"])
    P = w["pool"]
    # the graph pool: edges and four label vectors per graph in pinned memory
    pool = []
    for g in range(P):
        s_g = int(np.exp(rng.uniform(np.log(w["s_lo"]), np.log(w["s_hi"]))))
        n_g = max(s_g // 8, 16)
        if g % 2 == 0:
            scale = max(1, int(np.ceil(np.log2(n_g))))
            e = graphgen.rmat_edges_device(scale, n_g, 0, s_g, w["seed"] * 1000 + g, device=dev)
        else:
            kb = int(rng.integers(2, 65))
            e = graphgen.planted_edges_device(n_g, min(kb, n_g), s_g, 10.0,
                                              w["seed"] * 1000 + g, device=dev)
        eh = torch.empty((s_g, 2), dtype=torch.int32, pin_memory=True)
        eh.copy_(e)
        labs = []
        for j in range(4):
            K = int(rng.integers(w["K_lo"], w["K_hi"] + 1))
            yh = torch.empty(n_g, dtype=torch.int32, pin_memory=True)
            yh.copy_(graphgen.labels_device(n_g, K, w["seed"] * 7919 + 4 * g + j, device=dev))
            labs.append((K, yh.numpy()))
        kmax = max(K for K, _ in labs)
        out = torch.empty((n_g, kmax), dtype=torch.float32, pin_memory=True).numpy()
        pool.append(dict(s=s_g, n=n_g, edges=eh.numpy(), labs=labs, out=out))
        del e
    torch.cuda.synchronize()
    resident = list(range(0, P, P // w["resident"]))[: w["resident"]]
    kinds = rng.random(R) < w["relabel"]
    picks = [(int(rng.choice(resident)) if kinds[i] else int(rng.integers(P)),
              int(rng.integers(4))) for i in range(R)]
    edges_of = [pool[g]["s"] for g, _ in picks]
    total_edges = float(sum(edges_of))

    def zbuf(g, K):
        o = pool[g]["out"]
        return o.reshape(-1)[: pool[g]["n"] * K].reshape(pool[g]["n"], K)

    # plain: one synchronous call per request, graphs kept resident on the device
    dev_graphs = {}
    for g in resident:
        dev_graphs[g] = gee.Graph(torch.from_numpy(pool[g]["edges"]).to(dev), pool[g]["n"])
    service = np.empty(R)
    for warm in range(2):
        g, j = picks[warm]
        K, Y = pool[g]["labs"][j]
        gee.embed_host(pool[g]["edges"], Y, K, out=zbuf(g, K))
    for i, (g, j) in enumerate(picks):
        K, Y = pool[g]["labs"][j]
        t0 = time.perf_counter()
        if kinds[i]:
            dev_graphs[g].embed_host(Y, K, out=zbuf(g, K))
        else:
            gee.embed_host(pool[g]["edges"], Y, K, out=zbuf(g, K))
        service[i] = time.perf_counter() - t0
    plain_total = float(service.sum())
    # a few results to compare with the server's (copied before they are overwritten)
    check_ids = [i for i in range(R) if kinds[i]][:2] + [i for i in range(R) if not kinds[i]][:2]

    with gee.Server(hbm_budget_bytes=w["budget"], streams=w["streams"],
                    max_batch=w["max_batch"]) as srv:
        gid = {g: srv.add_graph(pool[g]["edges"], pool[g]["n"]) for g in resident}

        def submit(i):
            g, j = picks[i]
            K, Y = pool[g]["labs"][j]
            if kinds[i]:
                return srv.submit(Y, K, graph=gid[g], out=zbuf(g, K))
            return srv.submit(Y, K, edges=pool[g]["edges"], out=zbuf(g, K))

        # agreement with the plain path on a few requests
        worst = 0.0
        for i in check_ids:
            g, j = picks[i]
            K, Y = pool[g]["labs"][j]
            if kinds[i]:
                want = dev_graphs[g].embed_host(Y, K)
            else:
                want = gee.embed_host(pool[g]["edges"], Y, K)
            got, _ = srv.wait(submit(i))
            worst = max(worst, float(np.abs(got - want).max()))
        # burst: every request at once -> throughput
        t0 = time.perf_counter()
        tickets = [submit(i) for i in range(R)]
        for t in tickets:
            srv.wait(t)
        burst_s = time.perf_counter() - t0
        st_burst = srv.stats()
        # Poisson arrivals at load x the plain capacity -> latencies
        lam = w["load"] * R / plain_total
        arrivals = np.cumsum(rng.exponential(1.0 / lam, R))
        lat = np.empty(R)
        tickets = [None] * R
        ready = threading.Semaphore(0)

        def client():
            base = time.perf_counter()
            for i in range(R):
                d = base + arrivals[i] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = submit(i)
                ready.release()

        sampler = ClockSampler(local) if not args.no_clocks else None
        th = threading.Thread(target=client)
        t0 = time.perf_counter()
        th.start()
        for i in range(R):
            ready.acquire()
            _, lat[i] = srv.wait(tickets[i])
        th.join()
        stream_s = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        st = srv.stats()
    for g in dev_graphs.values():
        g.close()
    # plain latencies under the same arrivals: FIFO, one call at a time
    finish = 0.0
    plain_lat = np.empty(R)
    for i in range(R):
        start = max(arrivals[i], finish)
        finish = start + service[i]
        plain_lat[i] = (finish - arrivals[i]) * 1e3
    pct = lambda a, q: float(np.percentile(a, q))
    # bytes the burst moves over the host link (edges and labels in, Z out)
    h2d = sum((0 if kinds[i] else 8 * pool[g]["s"]) + 4 * pool[g]["n"]
              for i, (g, _) in enumerate(picks))
    d2h = sum(4 * pool[g]["n"] * pool[g]["labs"][j][0] for g, j in picks)
    link = _host_link_rates(dev)
    floor_s = max(h2d / (link["h2d_gbs"] * 1e9), d2h / (link["d2h_gbs"] * 1e9),
                  (h2d + d2h) / (link["both_gbs"] * 1e9))
    return {
        "requests": R, "total_edges": total_edges, "burst_s": burst_s,
        "config": {"workload": w["desc"], "requests": R,
                   "pool_graphs": P, "resident_graphs": len(resident),
                   "edges_total": total_edges, "budget_bytes": w["budget"],
                   "streams": w["streams"], "max_batch": w["max_batch"]},
        "plain": {"value": total_edges / plain_total, "seconds": plain_total,
                  "p50_ms": pct(plain_lat, 50), "p99_ms": pct(plain_lat, 99),
                  "api": "gee_embed_host / gee_embed_graph_host, one at a time"},
        "served": {"burst_seconds": burst_s, "edges_per_s": total_edges / burst_s,
                   "poisson_rate_per_s": lam, "load_vs_plain_capacity": w["load"],
                   "stream_seconds": stream_s, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                   "p50_ms_plain_same_arrivals": pct(plain_lat, 50),
                   "p99_ms_plain_same_arrivals": pct(plain_lat, 99)},
        "speedup_vs_plain": plain_total / burst_s,
        "h2d_bytes": h2d, "d2h_bytes": d2h,
        "host_link": dict(link, h2d_bytes=h2d, d2h_bytes=d2h, floor_seconds=floor_s,
                          burst_frac_of_floor=floor_s / burst_s),
        "max_abs_diff_vs_plain": worst,
        "server_stats": {"burst": st_burst, "end": st},
        "clocks": clocks,
    }


def run_serve(args, w, world, rank, local):
    """The serving workload's own JSON line (serve_measure on
    --requests requests)."""
    m = serve_measure(args, w, local, args.requests)
    R, total_edges, burst_s = m["requests"], m["total_edges"], m["burst_s"]
    line = {
        "metric": "serving: edges/s and p50/p99 latency vs sequential plain calls",
        "value": world * total_edges / burst_s, "unit": "edges/s", "n_gpus": world,
        "steps": R, "warmup": 2, "ms_per_step": burst_s * 1e3 / R,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": dict(m["config"], name=args.workload, parallelism="replicas"),
        "plain": m["plain"], "served": m["served"],
        "speedup_vs_plain": m["speedup_vs_plain"],
        "e2e": {"value": world * total_edges / burst_s, "unit": "edges/s",
                "h2d_bytes_per_step": m["h2d_bytes"] / R,
                "d2h_bytes_per_step": m["d2h_bytes"] / R},
        "host_link": m["host_link"],
        "max_abs_diff_vs_plain": m["max_abs_diff_vs_plain"],
        "server_stats": m["server_stats"],
        "clocks": m["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def _errors(got, z64, zref32=None):
    """Max abs / rel error of got against the FP64 values (rel over non-zero
    oracle cells; cells where the oracle is 0 must be exactly 0), and the max
    abs difference from RN32 of the exact quotient where it is known."""
    import numpy as np
    got = np.asarray(got, np.float64)
    nz = z64 != 0
    out = {"cells": int(got.size),
           "max_abs_err_vs_fp64": float(np.abs(got - z64).max()) if got.size else 0.0,
           "max_rel_err_vs_fp64": float((np.abs(got[nz] - z64[nz]) / np.abs(z64[nz])).max())
           if nz.any() else 0.0,
           "zeros_exact": bool(np.all(got[~nz] == 0))}
    if zref32 is not None:
        out["max_abs_diff_vs_rn32_exact"] = float(np.abs(got - zref32).max()) if got.size else 0.0
        out["bit_exact"] = bool(np.array_equal(np.asarray(got, np.float32), zref32))
    return out


def run_precision(args, w, world, rank, local):
    """The precision ladder: every arithmetic path against the FP64 oracle."""
    import numpy as np
    import torch

    import graphgen
    import oracle
    import paper_2402_04403_gb300 as gee
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(w["seed"])
    report = []

    def add(config, path, errs, **extra):
        report.append(dict({"config": config, "path": path}, **errs, **extra))

    # tiny SBM (the small parity workload): every row
    e, Y = graphgen.tiny_sbm(seed=1)
    K = 5
    wt = graphgen.weights(e.shape[0], seed=11)
    ed, yd, wd = (torch.from_numpy(a).to(dev) for a in (e, Y, wt))
    z64 = oracle.embed(e, Y, K)
    zr = oracle.embed_counts32(e, Y, K)
    for strat in ("atomic", "private", "segmented"):
        add("tiny SBM", f"uint32 counts ({strat})",
            _errors(gee.embed(ed, yd, K, strategy=strat).cpu().numpy(), z64, zr))
    z64w = oracle.embed(e, Y, K, weights=wt)
    add("tiny SBM + weights (0,1]", "FP32 weight sums (atomic)",
        _errors(gee.embed(ed, yd, K, weights=wd, strategy="atomic").cpu().numpy(), z64w))
    add("tiny SBM + weights (0,1]", "FP32 weight sums (segmented)",
        _errors(gee.embed(ed, yd, K, weights=wd, strategy="segmented").cpu().numpy(), z64w))
    add("tiny SBM + weights (0,1]", "fixed-point sums, FP64 division (deterministic)",
        _errors(gee.embed(ed, yd, K, weights=wd, deterministic=True).cpu().numpy(), z64w))
    z64l = oracle.embed(e, Y, K, weights=wt, laplacian=True)
    add("tiny SBM + weights (0,1]", "FP32 Laplacian (FP64 degree scale)",
        _errors(gee.embed(ed, yd, K, weights=wd, laplacian=True).cpu().numpy(), z64l))

    def sampled(config, edges_h, wts_h, Ys, K, graph, n, laplacian=False, multi=False,
                deterministic=False):
        """Rows: the 64 highest-degree nodes and random ones."""
        deg = np.bincount(edges_h.ravel(), minlength=n)
        rows = np.unique(np.concatenate([np.argsort(deg)[-64:],
                                         rng.integers(0, n, w["rows"])]))
        if multi:
            Z = graph.embed_multi(torch.from_numpy(Ys).to(dev), K).cpu().numpy()
            for l in (0, Ys.shape[0] - 1):
                r, z64r = oracle.embed_rows(edges_h, Ys[l], K, rows, weights=wts_h)
                add(config, f"multi-label FP32 (vector {l} of {Ys.shape[0]})",
                    _errors(Z[r, l * K:(l + 1) * K], z64r), rows_checked=int(r.size))
            return
        Yd = torch.from_numpy(Ys).to(dev)
        Z = graph.embed(Yd, K, laplacian=laplacian, deterministic=deterministic).cpu().numpy()
        if wts_h is None and not laplacian:
            r, z64r, C = oracle.embed_rows(edges_h, Ys, K, rows, with_counts=True)
            nk = oracle.class_counts(Ys, K)
            add(config, "uint32 counts (resident graph)",
                _errors(Z[r], z64r, oracle.round_counts(C, nk)), rows_checked=int(r.size))
        else:
            r, z64r = oracle.embed_rows(edges_h, Ys, K, rows, weights=wts_h, laplacian=laplacian)
            path = "FP32 Laplacian (resident graph)" if laplacian \
                else "FP32 weight sums (resident graph)"
            if deterministic:
                path = ("fixed-point Laplacian sums" if laplacian else "fixed-point sums") + \
                    ", FP64 division (resident graph, deterministic)"
            add(config, path, _errors(Z[r], z64r), rows_checked=int(r.size))

    # R-MAT scale 24 weighted (and the same graph with unit weights)
    W = WORKLOADS["rmat24"]
    n, s, K = W["n"], W["s"], W["K"]
    ed = graphgen.rmat_edges_device(W["scale"], n, 0, s, W["seed"], device=dev)
    wd = graphgen.weights_device(s, W["seed"] + 2, device=dev)
    Yd = graphgen.labels_device(n, K, W["seed"] + 1, W["frac_unlabeled"], device=dev)
    e_h, w_h, Y_h = ed.cpu().numpy(), wd.cpu().numpy(), Yd.cpu().numpy()
    with gee.Graph(ed, n, weights=wd) as g:
        sampled("R-MAT scale 24, weights (0,1]", e_h, w_h, Y_h, K, g, n)
        sampled("R-MAT scale 24, weights (0,1]", e_h, w_h, Y_h, K, g, n, laplacian=True)
        sampled("R-MAT scale 24, weights (0,1]", e_h, w_h, Y_h, K, g, n, deterministic=True)
        sampled("R-MAT scale 24, weights (0,1]", e_h, w_h, Y_h, K, g, n, laplacian=True,
                deterministic=True)
        Ys = np.stack([graphgen.labels(n, K, seed=900 + l, frac_unlabeled=0.1) for l in range(32)])
        sampled("R-MAT scale 24, weights (0,1], L=32", e_h, w_h, Ys, K, g, n, multi=True)
    with gee.Graph(ed, n) as g:
        sampled("R-MAT scale 24, unit weights", e_h, None, Y_h, K, g, n)
    # the one-shot edge-list call's weighted forms on the same rows: pushed
    # float atomics (sums in scheduling order) and binned records (float
    # sums with their rounding errors kept)
    deg = np.bincount(e_h.ravel(), minlength=n)
    rows = np.unique(np.concatenate([np.argsort(deg)[-64:], rng.integers(0, n, w["rows"])]))
    Z = torch.empty((n, K), dtype=torch.float32, device=dev)
    for lap in (False, True):
        r, z64r = oracle.embed_rows(e_h, Y_h, K, rows, weights=w_h, laplacian=lap)
        for strat in ("atomic", "binned"):
            gee.embed(ed, Yd, K, weights=wd, laplacian=lap, strategy=strat, out=Z)
            form = "Laplacian" if lap else "weight sums"
            path = (f"FP32 {form}, pushed atomics (one-shot ATOMIC)" if strat == "atomic"
                    else f"FP32 {form} with compensation (one-shot BINNED)")
            add("R-MAT scale 24, weights (0,1]", path,
                _errors(Z[torch.from_numpy(r).to(dev)].cpu().numpy(), z64r),
                rows_checked=int(r.size))
    del ed, wd, Yd, Z
    torch.cuda.empty_cache()
    # paper scale, unit weights (the headline workload)
    W = WORKLOADS["paper"]
    n, s, K = W["n"], W["s"], W["K"]
    ed = graphgen.rmat_edges_device(W["scale"], n, 0, s, W["seed"], device=dev)
    Yd = graphgen.labels_device(n, K, W["seed"] + 1, W["frac_unlabeled"], device=dev)
    e_h, Y_h = ed.cpu().numpy(), Yd.cpu().numpy()
    with gee.Graph(ed, n) as g:
        del ed
        sampled("paper scale (1.8B edges), unit weights", e_h, None, Y_h, K, g, n)
    line = {"metric": "max error vs the FP64 oracle, per arithmetic path",
            "value": max(r["max_rel_err_vs_fp64"] for r in report), "unit": "relative",
            "higher_is_better": False, "n_gpus": world, "steps": 1, "warmup": 0,
            "dtype": "u32/f32", "data": "synthetic",
            "config": {"workload": w["desc"], "name": args.workload}, "paths": report}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_unsup(args, w, world, rank, local):
    """Unsupervised GEE (gee_unsupervised) on a planted partition: rounds,
    nodes moved per round, time per round and agreement with the planted
    blocks."""
    import numpy as np
    import torch

    import graphgen
    import paper_2402_04403_gb300 as gee
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, s, K = w["n"], w["s"], w["K"]
    edges = graphgen.planted_edges_device(n, K, s, w["ratio"], w["seed"], device=dev)
    truth = graphgen.planted_labels_device(n, K, device=dev)
    noise = graphgen.labels_device(n, K, w["seed"] + 1, 0.0, device=dev)
    keep = graphgen.labels_device(n, 1 << 20, w["seed"] + 2, 0.0, device=dev) < int(
        w["known"] * (1 << 20))
    Y0 = torch.where(keep, truth, noise)
    g = gee.Graph(edges, n)
    del edges
    g.unsupervised(Y0, K, max_iter=1)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    e0.record(stream)
    y, Z, rounds, moved = g.unsupervised(Y0, K, max_iter=w["max_iter"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    gee.profile_read()
    gee.profile_enable(True)
    g.unsupervised(Y0, K, max_iter=2)
    torch.cuda.synchronize()
    gee.profile_enable(False)
    kernels = {k: {"launches": v["launches"], "ms": v["total_ms"] / max(v["launches"], 1)}
               for k, v in gee.profile_read().items()}
    # agreement: each found class counted by its most frequent planted block
    conf = torch.zeros(K * K, dtype=torch.int64, device=dev)
    conf.index_add_(0, (y.long() * K + truth.long()),
                    torch.ones(n, dtype=torch.int64, device=dev))
    conf = conf.view(K, K).cpu().numpy()
    purity = float(conf.max(axis=1).sum() / n)
    g.close()
    line = {
        "metric": "unsupervised GEE: time per round (embedding + k-means assignment)",
        "value": ms / max(rounds, 1), "unit": "ms/round", "higher_is_better": False,
        "n_gpus": world, "steps": rounds, "warmup": 1, "ms_per_step": ms / max(rounds, 1),
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64", "data": "synthetic",
        "config": {"workload": w["desc"], "name": args.workload, "n": n, "s": s, "K": K,
                   "max_iter": w["max_iter"], "parallelism": "replicas"},
        "rounds": rounds, "moved_per_round": moved, "total_ms": ms,
        "edges_per_s_per_round": s / (ms / max(rounds, 1) / 1e3),
        "purity_vs_planted_blocks": purity, "kernels_per_launch": kernels,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, w, world, rank, local):
    import torch

    import graphgen
    import paper_2402_04403_gb300 as gee
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, s, K = w["n"], w["s"], w["K"]

    t0 = time.perf_counter()
    edges = graphgen.rmat_edges_device(w["scale"], n, 0, s, w["seed"], device=dev)
    Y = graphgen.labels_device(n, K, w["seed"] + 1, w["frac_unlabeled"], device=dev)
    wts = graphgen.weights_device(s, w["seed"] + 2, device=dev) if w["weighted"] else None
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    t0 = time.perf_counter()
    g = gee.Graph(edges, n, weights=wts)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t0
    info = g.info()
    lap = w["laplacian"]
    Z = torch.empty((n, K), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        g.embed(Y, K, laplacian=lap, out=Z)
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if not args.no_clocks else None
    barrier(world)
    torch.cuda.synchronize()
    gee.profile_read()  # drop warm-up records
    gee.profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.embed(Y, K, laplacian=lap, out=Z)
    ev1.record(stream)
    torch.cuda.synchronize()
    gee.profile_enable(False)
    barrier(world)
    clocks = sampler.stop() if sampler else None
    prof = gee.profile_read()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world)
    ms_per_step = ms_max / args.steps
    value = world * s / (ms_per_step / 1e3)

    peak, peak_kind = measured_peaks()
    pass_kernels = ("k_pull_light", "k_pull_heavy", "k_hub_fixup")
    pass_ms = sum(prof[k]["total_ms"] / max(1, prof[k]["launches"])
                  for k in pass_kernels if k in prof)
    achieved = pull_bytes(w) / (pass_ms / 1e3) / 1e9
    step_gbs = algorithmic_bytes(w) / (ms_per_step / 1e3) / 1e9
    launches = sum(v["launches"] for v in prof.values())
    heavy_arcs, light_arcs = info["hub_arcs"], 2 * s - info["hub_arcs"]
    kernel_bytes = {  # compulsory bytes each pass kernel must move
        "k_pull_light": 4 * light_arcs * (1 + w["weighted"]) + n + 4 * n * K,
        "k_pull_heavy": 4 * heavy_arcs * (1 + w["weighted"]),
    }
    result = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if (w["weighted"] or lap) else "u32", "data": "synthetic",
        "config": config_for(args, w),
        "roofline": {"bound": "hbm",
                     "kernel": "edge pass: k_pull_light + k_pull_heavy + k_hub_fixup",
                     "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "traffic": ncu_traffic("k_pull", args.workload)
                     if not args.scale_shift else None,
                     "algorithmic_bytes_per_launch": pull_bytes(w),
                     "avg_launch_ms": pass_ms,
                     "step_algorithmic_bytes": algorithmic_bytes(w),
                     "step_gbs": step_gbs, "step_frac": step_gbs / peak,
                     "frac_of_nominal_8tbs": step_gbs / 8000.0,
                     # the looser reading: also two 4-byte label gathers per edge
                     "loose_bytes_per_step": algorithmic_bytes(w) + 8 * s,
                     "loose_frac": (algorithmic_bytes(w) + 8 * s)
                     / (ms_per_step * 1e-3) / 1e9 / peak,
                     "gather_bound": gather_bound(g, w["K"], prof, clocks)},
        "kernels": {k: dict({"launches": v["launches"],
                             "avg_ms": v["total_ms"] / max(1, v["launches"])},
                            **({"gbs": kernel_bytes[k] / (v["total_ms"] / max(1, v["launches"]))
                                / 1e6} if k in kernel_bytes else {}))
                    for k, v in prof.items()},
        "gpu_launches": launches,
        "clocks": clocks,
        "ingest": {"graph_build_s": ingest_s, "generate_s": gen_s,
                   "hub_rows": info["hub_rows"], "hub_arcs": info["hub_arcs"],
                   "graph_device_bytes": info["device_bytes"]},
    }

    if not args.no_e2e:
        Yh = Y.cpu().pin_memory()
        Zh = torch.empty((n, K), dtype=torch.float32).pin_memory()
        g.embed_host(Yh, K, laplacian=lap, out=Zh)
        barrier(world)
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            g.embed_host(Yh, K, laplacian=lap, out=Zh)
        e2e_s = max_over_ranks(time.perf_counter() - t, world) / args.e2e_steps
        result["e2e"] = {"value": world * s / e2e_s, "unit": "edges/s",
                         "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n * K,
                         "ms_per_step": 1e3 * e2e_s,
                         "api": "gee_embed_graph_host (pinned host Y and Z)"}
        del Zh, Yh

    if not args.no_oneshot:
        g_close_first = args.workload.startswith("paper")
        if g_close_first:
            g.close()  # free the CSR so the one-shot scratch fits comfortably
        gee.embed(edges, Y, K, weights=wts, laplacian=lap, out=Z)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.oneshot_steps):
            gee.embed(edges, Y, K, weights=wts, laplacian=lap, out=Z)
        e1.record(stream)
        torch.cuda.synchronize()
        os_ms = e0.elapsed_time(e1) / args.oneshot_steps
        result["oneshot"] = {"value": s / (os_ms / 1e3), "unit": "edges/s",
                             "ms_per_step": os_ms,
                             "strategy": gee.pick_strategy(s, n, K),
                             "api": "gee_embed (edge list in, Z out, nothing resident)"}
        # per-kernel times of one traced call (CUDA events on the stream)
        gee.profile_read()
        gee.profile_enable(True)
        gee.embed(edges, Y, K, weights=wts, laplacian=lap, out=Z)
        torch.cuda.synchronize()
        result["oneshot"]["kernels"] = {
            k: round(v["total_ms"], 3) for k, v in gee.profile_read().items()}
        gee.profile_enable(False)
        if not g_close_first or result["oneshot"]["strategy"] == "binned":
            # another one-shot strategy: the pushed atomics, or a temporary
            # CSR and the pull pass
            other = ("atomic" if result["oneshot"]["strategy"] == "binned" else
                     "segmented" if result["oneshot"]["strategy"] != "segmented" else "atomic")
            gee.embed(edges, Y, K, weights=wts, laplacian=lap, out=Z, strategy=other)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.oneshot_steps):
                gee.embed(edges, Y, K, weights=wts, laplacian=lap, out=Z, strategy=other)
            e1.record(stream)
            torch.cuda.synchronize()
            o_ms = e0.elapsed_time(e1) / args.oneshot_steps
            result["oneshot_" + other] = {"value": s / (o_ms / 1e3), "unit": "edges/s",
                                          "ms_per_step": o_ms}
    g.close()

    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(w, True, shift=args.cpu_shift)
    if (args.workload == "paper" and world == 1 and args.serve_requests > 0
            and not args.no_serve):
        # the metric's second half: serving p50/p99 beside plain calls, on
        # the serving workload's request mix (the paper graph freed first)
        del edges, Y, Z, wts
        torch.cuda.empty_cache()
        ws = dict(WORKLOADS["serve"])
        if args.serve_streams:
            ws["streams"] = args.serve_streams
        if args.serve_batch:
            ws["max_batch"] = args.serve_batch
        m = serve_measure(args, ws, local, args.serve_requests)
        result["serving"] = {
            "requests": m["requests"], "workload": ws["desc"],
            "edges_per_s": m["served"]["edges_per_s"],
            "plain_edges_per_s": m["plain"]["value"],
            "speedup_vs_plain": m["speedup_vs_plain"],
            "p50_ms": m["served"]["p50_ms"], "p99_ms": m["served"]["p99_ms"],
            "plain_p50_ms": m["served"]["p50_ms_plain_same_arrivals"],
            "plain_p99_ms": m["served"]["p99_ms_plain_same_arrivals"],
            "load_vs_plain_capacity": m["served"]["load_vs_plain_capacity"],
            "host_link": {k: m["host_link"][k] for k in
                          ("h2d_gbs", "d2h_gbs", "both_gbs", "floor_seconds",
                           "burst_frac_of_floor")},
            "max_concurrent_groups": m["server_stats"]["end"]["max_concurrent"],
            "max_abs_diff_vs_plain": m["max_abs_diff_vs_plain"],
        }
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="paper")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--oneshot-steps", type=int, default=3)
    ap.add_argument("--cpu-shift", type=int, default=5,
                    help="cpu_baseline sample = workload / 2^shift")
    ap.add_argument("--scale-shift", type=int, default=0,
                    help="shrink the workload by 2^shift (same generator; for profiling)")
    ap.add_argument("--requests", type=int, default=10000,
                    help="serve workload: number of requests")
    ap.add_argument("--serve-streams", type=int, default=0,
                    help="serve workload: server slots (0: the workload's)")
    ap.add_argument("--serve-batch", type=int, default=0,
                    help="serve workload: requests per group (0: the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oneshot", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="paper workload: skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="paper workload: requests of the serving measurement")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    w = dict(WORKLOADS[args.workload])
    if args.serve_streams:
        w["streams"] = args.serve_streams
    if args.serve_batch:
        w["max_batch"] = args.serve_batch
    if args.scale_shift and "graphs" not in w and "pool" not in w and \
            args.workload not in ("precision", "unsup"):
        sh = args.scale_shift
        w.update(scale=w["scale"] - sh, n=w["n"] >> sh, s=w["s"] >> sh,
                 desc=w["desc"] + f" (shrunk by 2^{sh}: n={w['n'] >> sh}, s={w['s'] >> sh})")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, w, world, rank)
    elif w.get("L", 1) > 1:
        run_multi(args, w, world, rank, local)
    elif "graphs" in w:
        run_batch(args, w, world, rank, local)
    elif "pool" in w:
        run_serve(args, w, world, rank, local)
    elif args.workload == "precision":
        run_precision(args, w, world, rank, local)
    elif args.workload == "unsup":
        run_unsup(args, w, world, rank, local)
    else:
        run_ours(args, w, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
