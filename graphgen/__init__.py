"""Seeded synthetic graph inputs: R-MAT and SBM edge lists, labels, weights.

This module only draws random inputs; it holds none of the embedding's
arithmetic.  It is the one piece of code that both the oracle side and the GPU
side of the test suite consume.

Every random number comes from the counter-based generator Philox4x32-10
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), so any single edge, label or weight is a pure function of
(seed, index).  The host implementation here (numpy) and the device
implementation in ``graphgen.cu`` compute the same values bit for bit; a test
checks that on samples.  Large graphs are drawn on the device; small ones on
the host.

Counter layout of one Philox call: (index_lo, index_hi, word2, tag) with the
64-bit seed as key.  ``tag`` separates the streams below.

R-MAT (Chakrabarti, Zhan, Faloutsos, SDM'04): each edge picks one quadrant per
level with probabilities (a, b, c, 1-a-b-c) using 16-bit uniforms
(thresholds round(p * 65536)), most significant bit first; node ids are then
mapped through a keyed bijection of [0, 2^scale) (Graph500-style relabeling,
so that hubs are not clustered at small ids).  When n < 2^scale an edge with
an endpoint >= n is redrawn with the next attempt number (word2 carries
attempt * 8 + call); after 64 attempts the endpoints are reduced modulo n.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

TAG_RMAT = 0x524D4154     # "RMAT"
TAG_PERM = 0x5045524D     # "PERM"
TAG_LABEL = 0x4C41424C    # "LABL"
TAG_WEIGHT = 0x57474854   # "WGHT"
TAG_SBM = 0x53424D30      # "SBM0"
TAG_SHUFFLE = 0x53484646  # "SHFF"
TAG_PLANTED = 0x504C4E54  # "PLNT"

RMAT_MAX_ATTEMPTS = 64
# elements per host batch: keeps the Philox temporaries cache-sized
_HOST_CHUNK = 1 << 14
# odd multipliers of the id bijection (any odd constants work)
_PERM_MUL1 = 0x2545F491
_PERM_MUL2 = 0x9E3779B1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on numpy arrays (broadcast).  Returns four
    uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK32
                      for x in np.broadcast_arrays(c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r != 9:
            k0 = (k0 + _W0) & MASK32
            k1 = (k1 + _W1) & MASK32
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def _words(idx, word2, tag, seed):
    idx = np.asarray(idx, dtype=np.uint64)
    k0, k1 = _key(seed)
    return philox4x32_10(idx & MASK32, idx >> np.uint64(32), word2, tag, k0, k1)


# ----------------------------------------------------------------------------
# R-MAT
# ----------------------------------------------------------------------------
def rmat_thresholds(a, b, c):
    A = int(round(a * 65536))
    AB = int(round((a + b) * 65536))
    ABC = int(round((a + b + c) * 65536))
    if not (0 <= A <= AB <= ABC <= 65536):
        raise ValueError("R-MAT probabilities must be non-negative and sum <= 1")
    return A, AB, ABC


def perm_keys(seed):
    w = _words(np.zeros(1, np.uint64), 0, TAG_PERM, seed)
    return int(w[0][0]), int(w[1][0])


def permute_ids(x, scale, seed):
    """Keyed bijection of [0, 2^scale): xor, multiply by odd, xorshift, twice."""
    mask = np.uint64((1 << scale) - 1)
    h = np.uint64(max(1, scale // 2))
    ka, kb = perm_keys(seed)
    x = np.asarray(x, dtype=np.uint64)
    x = (x ^ np.uint64(ka)) & mask
    x = (x * np.uint64(_PERM_MUL1)) & mask
    x ^= x >> h
    x = (x * np.uint64(_PERM_MUL2)) & mask
    x ^= x >> h
    x = (x ^ np.uint64(kb)) & mask
    return x


def _rmat_attempt(idx, attempt, scale, thr, seed):
    A, AB, ABC = (np.uint32(t) for t in thr)
    u = np.zeros(idx.shape, np.uint64)
    v = np.zeros(idx.shape, np.uint64)
    ncalls = (scale + 7) // 8
    for call in range(ncalls):
        w = _words(idx, attempt * 8 + call, TAG_RMAT, seed)
        for j in range(8):
            level = call * 8 + j
            if level >= scale:
                break
            r = (w[j // 2] >> np.uint32(16 * (j % 2))) & np.uint32(0xFFFF)
            ub = (r >= AB).astype(np.uint64)          # quadrants c, d: row bit 1
            vb = (((r >= A) & (r < AB)) | (r >= ABC)).astype(np.uint64)
            u = (u << np.uint64(1)) | ub
            v = (v << np.uint64(1)) | vb
    return permute_ids(u, scale, seed), permute_ids(v, scale, seed)


def _in_chunks(fn, start, count, out):
    """Fill out[0:count] with fn(start + i, m) over consecutive batches of
    at most _HOST_CHUNK elements (every element is a pure function of its
    index, so the batching does not change any value)."""
    for i in range(0, count, _HOST_CHUNK):
        m = min(_HOST_CHUNK, count - i)
        out[i:i + m] = fn(start + i, m)
    return out


def rmat_edges(scale, n, start, count, seed, a=0.57, b=0.19, c=0.19):
    """Edges [start, start+count) of the seeded R-MAT graph, (count, 2) int32."""
    if n > (1 << scale) or n < 1:
        raise ValueError("need 1 <= n <= 2^scale")
    thr = rmat_thresholds(a, b, c)
    return _in_chunks(lambda st, m: _rmat_block(scale, n, st, m, seed, thr),
                      start, count, np.empty((count, 2), np.int32))


def _rmat_block(scale, n, start, count, seed, thr):
    idx = np.arange(start, start + count, dtype=np.uint64)
    out_u = np.zeros(count, np.uint64)
    out_v = np.zeros(count, np.uint64)
    todo = np.arange(count)
    nn = np.uint64(n)
    for attempt in range(RMAT_MAX_ATTEMPTS):
        if todo.size == 0:
            break
        u, v = _rmat_attempt(idx[todo], attempt, scale, thr, seed)
        ok = (u < nn) & (v < nn)
        out_u[todo[ok]] = u[ok]
        out_v[todo[ok]] = v[ok]
        if attempt == RMAT_MAX_ATTEMPTS - 1:
            bad = todo[~ok]
            out_u[bad] = u[~ok] % nn
            out_v[bad] = v[~ok] % nn
        todo = todo[~ok]
    return np.stack([out_u, out_v], axis=1).astype(np.int32)


# ----------------------------------------------------------------------------
# labels and weights
# ----------------------------------------------------------------------------
def unlabeled_threshold(frac_unlabeled):
    return min(int(frac_unlabeled * 4294967296.0), 4294967296)


def labels(n, K, seed, frac_unlabeled=0.0, start=0):
    """Y[i] uniform in [0, K), or -1 with probability frac_unlabeled."""
    return _in_chunks(lambda st, m: _labels_block(m, K, seed, frac_unlabeled, st),
                      start, n, np.empty(n, np.int32))


def _labels_block(n, K, seed, frac_unlabeled, start):
    idx = np.arange(start, start + n, dtype=np.uint64)
    w = _words(idx, 0, TAG_LABEL, seed)
    cls = ((w[1].astype(np.uint64) * np.uint64(K)) >> np.uint64(32)).astype(np.int32)
    thr = unlabeled_threshold(frac_unlabeled)
    if thr > 0:
        cls[w[0].astype(np.uint64) < np.uint64(thr)] = -1
    return cls


def weights(s, seed, start=0):
    """w[i] = (top 24 bits + 1) / 2^24, uniform on (0, 1], exact in float32."""
    return _in_chunks(lambda st, m: _weights_block(m, seed, st),
                      start, s, np.empty(s, np.float32))


def _weights_block(s, seed, start):
    idx = np.arange(start, start + s, dtype=np.uint64)
    w = _words(idx, 0, TAG_WEIGHT, seed)
    return (((w[0] >> np.uint32(8)).astype(np.float64) + 1.0) / 16777216.0
            ).astype(np.float32)


# ----------------------------------------------------------------------------
# stochastic block model (host only; small graphs)
# ----------------------------------------------------------------------------
def sbm(block_sizes, p_in, p_out, seed, shuffle=True):
    """Undirected SBM without self-loops: every pair u < v is an edge with
    probability p_in (same block) or p_out.  Returns (edges (s,2) int32,
    block labels int32).  Pair (u, v) in block pair (i, j) uses Philox word
    (t mod 4) of call t // 4, t the pair's index in the block rectangle."""
    sizes = [int(x) for x in block_sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    nb = len(sizes)
    chunks = []
    for i in range(nb):
        for j in range(i, nb):
            p = p_in if i == j else p_out
            thr = np.uint64(min(int(p * 4294967296.0), 4294967295))
            mi, mj = sizes[i], sizes[j]
            total = mi * mj
            ncalls = (total + 3) // 4
            step = 1 << 21
            for c0 in range(0, ncalls, step):
                calls = np.arange(c0, min(ncalls, c0 + step), dtype=np.uint64)
                words = _words(calls, i * nb + j, TAG_SBM, seed)
                r = np.stack(words, axis=1).ravel()   # trial t = 4*call + word
                t = np.uint64(4 * c0) + np.flatnonzero(r < np.uint32(thr)
                                                       ).astype(np.uint64)
                hit = t[t < np.uint64(total)]
                a = (hit // np.uint64(mj)).astype(np.int64)
                b = (hit % np.uint64(mj)).astype(np.int64)
                if i == j:
                    keep = a < b
                    a, b = a[keep], b[keep]
                chunks.append(np.stack([a + offs[i], b + offs[j]], axis=1))
    e = (np.concatenate(chunks) if chunks else np.zeros((0, 2), np.int64))
    e = e.astype(np.int32)
    if shuffle and e.shape[0] > 1:
        key = _words(np.arange(e.shape[0], dtype=np.uint64), 0, TAG_SHUFFLE, seed)
        order = np.argsort((key[0].astype(np.uint64) << np.uint64(32))
                           | key[1].astype(np.uint64), kind="stable")
        e = e[order]
    y = np.repeat(np.arange(nb, dtype=np.int32), sizes)
    return np.ascontiguousarray(e), y


def tiny_sbm(seed=1):
    """The 5-block SBM of the small parity workload: 5 x 2000 nodes,
    p_in = 0.02, p_out = 0.002, labels = blocks, K = 5."""
    return sbm([2000] * 5, 0.02, 0.002, seed)


def planted_block_start(g, n, K):
    """First node of block g when n nodes are cut into K nearly equal blocks
    (node i is in block floor(i K / n))."""
    return (np.asarray(g, dtype=np.int64) * n + K - 1) // K


def planted_labels(n, K):
    """Block of every node: floor(i K / n)."""
    return ((np.arange(n, dtype=np.int64) * K) // n).astype(np.int32)


def planted_same_threshold(n, K, ratio):
    """2^32 times the probability that an edge stays inside its first
    endpoint's block, for p_in / p_out = ratio: ratio (b-1) / (ratio (b-1) +
    n - b) with b = n / K, the share of a node's expected SBM edges that are
    inside its block."""
    b = n / K
    inside = ratio * (b - 1.0)
    q = 1.0 if n - b <= 0 else (inside / (inside + (n - b)) if inside > 0 else 0.0)
    return min(int(q * 4294967296.0), 1 << 32)


def planted_edges(n, K, s, ratio, seed, start=0):
    """Edges [start, start+s) of a planted-partition graph drawn edge by
    edge: the first endpoint uniform over the n nodes, the second inside its
    block with probability planted_same_threshold / 2^32 (else uniform over
    the other blocks).  The edge-sampling form of a K-block SBM with
    p_in / p_out = ratio, for graphs too large to draw pair by pair.
    (s, 2) int32."""
    idx = np.arange(start, start + s, dtype=np.uint64)
    x, y, z, _ = _words(idx, 0, TAG_PLANTED, seed)
    nn = np.uint64(n)
    u = (x.astype(np.uint64) * nn) >> np.uint64(32)
    g = (u * np.uint64(K)) // nn
    b0 = (g * nn + np.uint64(K - 1)) // np.uint64(K)
    b1 = ((g + np.uint64(1)) * nn + np.uint64(K - 1)) // np.uint64(K)
    size = b1 - b0
    z64 = z.astype(np.uint64)
    v_in = b0 + ((z64 * size) >> np.uint64(32))
    r = (z64 * (nn - size)) >> np.uint64(32)
    v_out = np.where(r < b0, r, r + size)
    same = y.astype(np.uint64) < np.uint64(planted_same_threshold(n, K, ratio))
    v = np.where(same, v_in, v_out)
    return np.stack([u, v], axis=1).astype(np.int32)


def random_graph(n, s, seed, self_loops=True):
    """Uniform random multigraph with s edges on n nodes (small tests)."""
    idx = np.arange(s, dtype=np.uint64)
    w = _words(idx, 0, TAG_RMAT ^ 0xFF, seed)
    u = ((w[0].astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    v = ((w[1].astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    if not self_loops:
        v = np.where(u == v, (v + 1) % max(n, 1), v)
    return np.stack([u, v], axis=1).astype(np.int32)


# ----------------------------------------------------------------------------
# device generation (graphgen.cu): the same values, drawn on the GPU
# ----------------------------------------------------------------------------
import ctypes as _ctypes
import os as _os
import subprocess as _subprocess
import threading as _threading

_HERE = _os.path.dirname(_os.path.abspath(__file__))
_CU = _os.path.join(_HERE, "graphgen.cu")
_SO = _os.path.join(_HERE, "libgraphgen.so")
_lock = _threading.Lock()
_dev_lib = None


def build(force=False):
    """Compile graphgen.cu into libgraphgen.so (sm_103a) in place."""
    if force or not _os.path.exists(_SO) or _os.path.getmtime(_SO) < _os.path.getmtime(_CU):
        nvcc = _os.environ.get("NVCC") or "nvcc"
        tmp = _SO + f".tmp{_os.getpid()}"
        _subprocess.check_call([
            nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-shared",
            "-cudart", "static", "-Xlinker", "--exclude-libs,ALL", "-o", tmp, _CU])
        _os.replace(tmp, _SO)
    return _SO


def _lib():
    global _dev_lib
    with _lock:
        if _dev_lib is None:
            lib = _ctypes.CDLL(build())
            P, I64, I32, U32, U64 = (_ctypes.c_void_p, _ctypes.c_int64, _ctypes.c_int32,
                                     _ctypes.c_uint32, _ctypes.c_uint64)
            lib.graphgen_rmat.argtypes = [P, I64, I64, _ctypes.c_int, I64, U32, U32, U32, U64, P]
            lib.graphgen_labels.argtypes = [P, I64, I64, I32, U64, U64, P]
            lib.graphgen_weights.argtypes = [P, I64, I64, U64, P]
            lib.graphgen_planted.argtypes = [P, I64, I64, I64, I32, U64, U64, P]
            lib.graphgen_planted_labels.argtypes = [P, I64, I32, P]
            for f in (lib.graphgen_rmat, lib.graphgen_labels, lib.graphgen_weights,
                      lib.graphgen_planted, lib.graphgen_planted_labels):
                f.restype = _ctypes.c_int
            _dev_lib = lib
    return _dev_lib


def _stream():
    import torch
    return _ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def rmat_edges_device(scale, n, start, count, seed, a=0.57, b=0.19, c=0.19,
                      out=None, device="cuda"):
    """Same edges as rmat_edges, drawn on the GPU into an int32 (count, 2) tensor."""
    import torch
    if out is None:
        out = torch.empty((count, 2), dtype=torch.int32, device=device)
    A, AB, ABC = rmat_thresholds(a, b, c)
    rc = _lib().graphgen_rmat(_ctypes.c_void_p(out.data_ptr()), start, count, scale, n,
                              A, AB, ABC, int(seed) & 0xFFFFFFFFFFFFFFFF, _stream())
    if rc != 0:
        raise RuntimeError(f"graphgen_rmat failed ({rc})")
    return out


def labels_device(n, K, seed, frac_unlabeled=0.0, start=0, out=None, device="cuda"):
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=device)
    rc = _lib().graphgen_labels(_ctypes.c_void_p(out.data_ptr()), start, n, K,
                                unlabeled_threshold(frac_unlabeled),
                                int(seed) & 0xFFFFFFFFFFFFFFFF, _stream())
    if rc != 0:
        raise RuntimeError(f"graphgen_labels failed ({rc})")
    return out


def weights_device(s, seed, start=0, out=None, device="cuda"):
    import torch
    if out is None:
        out = torch.empty(s, dtype=torch.float32, device=device)
    rc = _lib().graphgen_weights(_ctypes.c_void_p(out.data_ptr()), start, s,
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, _stream())
    if rc != 0:
        raise RuntimeError(f"graphgen_weights failed ({rc})")
    return out


def planted_edges_device(n, K, s, ratio, seed, start=0, out=None, device="cuda"):
    """Same edges as planted_edges, drawn on the GPU."""
    import torch
    if out is None:
        out = torch.empty((s, 2), dtype=torch.int32, device=device)
    rc = _lib().graphgen_planted(_ctypes.c_void_p(out.data_ptr()), start, s, n, K,
                                 planted_same_threshold(n, K, ratio),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, _stream())
    if rc != 0:
        raise RuntimeError(f"graphgen_planted failed ({rc})")
    return out


def planted_labels_device(n, K, out=None, device="cuda"):
    """Same labels as planted_labels, written on the GPU."""
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=device)
    rc = _lib().graphgen_planted_labels(_ctypes.c_void_p(out.data_ptr()), n, K, _stream())
    if rc != 0:
        raise RuntimeError(f"graphgen_planted_labels failed ({rc})")
    return out
