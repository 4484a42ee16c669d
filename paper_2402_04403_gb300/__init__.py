"""GB300-native One-Hot Graph Encoder Embedding (GEE).

Python binding of libgee.so (include/gee.h): the functions below check and
marshal PyTorch tensors (device memory, streams) and call the C ABI; every
step of the embedding -- label check and histogram, edge pass, scaling --
runs in the library's CUDA kernels.  Method: Algorithm 1 of "Edge-Parallel
Graph Encoder Embedding" (arXiv 2402.04403): Z = A W with
W(i, Y(i)) = 1 / count(Y = Y(i)).

Conventions: ``edges`` int32 (s, 2) of (u, v); ``weights`` float32 (s,) or
None for unit weights; ``Y`` int32 (n,) with classes 0..K-1 and -1 for
"class unknown"; result ``Z`` float32 (n, K).
"""
from __future__ import annotations

import ctypes

from . import _lib as _lib_mod
from ._lib import (GeeError, HUB_DEGREE, MAX_CLASSES, NOALLOC_MAX_NODES, STATUS, STATUS_NAMES,
                   STRATEGIES, STRATEGY_NAMES, KernelTime, check, lib, options)

__all__ = ["GeeError", "Graph", "embed", "embed_host", "histogram",
           "pick_strategy", "workspace_bytes", "debug_fail_allocs", "status_string", "STATUS",
           "STRATEGIES", "MAX_CLASSES", "HUB_DEGREE", "load", "profile_enable",
           "profile_read", "embed_noalloc", "NOALLOC_MAX_NODES", "embed_batch",
           "Server", "autotune", "tune_table", "tune_set"]


def load():
    """Load libgee.so now (raises if it is missing)."""
    return lib()


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, name, shape=None):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() > 0 else None


def _edges_shape(edges):
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must have shape (s, 2)")
    return edges.shape[0]


def profile_enable(on: bool = True) -> None:
    """Start/stop CUDA-event tracing of every library kernel launch."""
    lib().gee_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{kernel name: {"launches", "total_ms", "max_ms"}} since the last read."""
    buf = (KernelTime * 64)()
    got = lib().gee_profile_read(buf, len(buf))
    out = {}
    for i in range(min(got, len(buf))):
        t = buf[i]
        out[t.name.decode()] = {"launches": int(t.launches), "total_ms": float(t.total_ms),
                                "max_ms": float(t.max_ms)}
    return out


def status_string(code: int) -> str:
    return lib().gee_status_string(int(code)).decode()


def histogram(Y, K: int, stream=None):
    """Class sizes n_k (int32 tensor of length K; the library writes uint32)."""
    torch = _torch()
    n = Y.numel()
    counts = torch.empty(K, dtype=torch.int32, device=Y.device)
    rc = lib().gee_histogram(_dev_ptr(Y, torch.int32, "Y"), n, int(K),
                             ctypes.c_void_p(counts.data_ptr()), _stream_handle(stream))
    check(rc, "gee_histogram")
    return counts


def debug_fail_allocs(count: int) -> None:
    """Test hook (gee_debug_fail_allocs): the next ``count`` device
    allocations of the library fail as if the device were out of memory."""
    lib().gee_debug_fail_allocs(int(count))


def pick_strategy(s: int, n: int, K: int, strategy="auto", private_max_cells=0) -> str:
    o = options(strategy, True, private_max_cells)
    return STRATEGY_NAMES[lib().gee_pick_strategy(int(s), int(n), int(K), ctypes.byref(o))]


def workspace_bytes(s, n, K, weighted=False, laplacian=False, strategy="auto") -> int:
    o = options(strategy)
    return int(lib().gee_workspace_bytes(int(s), int(n), int(K), int(bool(weighted)),
                                         int(bool(laplacian)), ctypes.byref(o)))


def embed(edges, Y, K: int, weights=None, laplacian: bool = False, *,
          strategy="auto", validate_edges: bool = True, block: int = 0,
          private_max_cells: int = 0, deterministic: bool = False, out=None,
          stream=None):
    """Z = A W for a device edge list (gee_embed).  deterministic: float
    sums in fixed point, bitwise reproducible (the SEGMENTED form)."""
    torch = _torch()
    s = _edges_shape(edges)
    n = Y.numel()
    if out is None:
        out = torch.empty((n, K), dtype=torch.float32, device=Y.device)
    o = options(strategy, validate_edges, private_max_cells, block, deterministic)
    rc = lib().gee_embed(
        _dev_ptr(edges, torch.int32, "edges"),
        _dev_ptr(weights, torch.float32, "weights", (s,)),
        s, _dev_ptr(Y, torch.int32, "Y", (n,)), n, int(K), int(bool(laplacian)),
        _dev_ptr(out, torch.float32, "out", (n, K)), ctypes.byref(o),
        _stream_handle(stream))
    check(rc, "gee_embed")
    return out


def embed_batch(problems, *, validate_edges: bool = True, strategy="auto", stream=None,
                raise_on_error: bool = True):
    """gee_embed_batch: many independent problems in one launch sequence.

    ``problems``: sequence of dicts with keys ``edges`` (int32 (s, 2) CUDA
    tensor), ``Y`` (int32 (n,)), ``K`` and optionally ``weights`` (float32
    (s,)) and ``out`` (float32 (n, K)).  Returns the list of Z tensors, or
    (Zs, statuses) with ``raise_on_error=False``."""
    torch = _torch()
    arr = (_lib_mod.Problem * max(len(problems), 1))()
    outs = []
    for i, q in enumerate(problems):
        edges, Y, K = q["edges"], q["Y"], int(q["K"])
        s = _edges_shape(edges)
        n = Y.numel()
        out = q.get("out")
        if out is None:
            out = torch.empty((n, K), dtype=torch.float32, device=Y.device)
        outs.append(out)
        arr[i].edges = _dev_ptr(edges, torch.int32, "edges")
        arr[i].weights = _dev_ptr(q.get("weights"), torch.float32, "weights", (s,))
        arr[i].s = s
        arr[i].Y = _dev_ptr(Y, torch.int32, "Y", (n,))
        arr[i].n = n
        arr[i].K = K
        arr[i].reserved = 0
        arr[i].Z = _dev_ptr(out, torch.float32, "out", (n, K))
    statuses = (ctypes.c_int * max(len(problems), 1))()
    o = options(strategy, validate_edges=validate_edges)
    rc = lib().gee_embed_batch(arr, len(problems), statuses, ctypes.byref(o),
                               _stream_handle(stream))
    codes = [int(statuses[i]) for i in range(len(problems))]
    if raise_on_error:
        check(rc, "gee_embed_batch")
        return outs
    return outs, codes


def tune_table() -> list:
    """The current device's GEE_AUTO tuning table (empty if not tuned)."""
    count = lib().gee_tune_get(None, 0)
    buf = (_lib_mod.TuneCell * max(count, 1))()
    got = lib().gee_tune_get(buf, count)
    out = []
    for i in range(min(got, count)):
        c = buf[i]
        out.append({"log2_cells": c.log2_cells, "log2_density": c.log2_density,
                    "strategy": STRATEGY_NAMES[c.strategy], "block": c.block,
                    "ms_atomic": c.ms_atomic, "ms_private": c.ms_private,
                    "ms_segmented": c.ms_segmented})
    return out


def tune_set(table) -> None:
    """Install a tuning table (as returned by tune_table); [] resets."""
    buf = (_lib_mod.TuneCell * max(len(table), 1))()
    for i, c in enumerate(table):
        buf[i].log2_cells = int(c["log2_cells"])
        buf[i].log2_density = int(c["log2_density"])
        st = c["strategy"]
        buf[i].strategy = STRATEGIES[st] if isinstance(st, str) else int(st)
        buf[i].block = int(c.get("block", 0))
        buf[i].ms_atomic = float(c.get("ms_atomic", -1))
        buf[i].ms_private = float(c.get("ms_private", -1))
        buf[i].ms_segmented = float(c.get("ms_segmented", -1))
    check(lib().gee_tune_set(buf, len(table)), "gee_tune_set")


def autotune(effort: int = 0, stream=None) -> list:
    """gee_autotune: time the edge-list strategies on this device and
    install the fastest per problem shape for GEE_AUTO; returns the table."""
    check(lib().gee_autotune(int(effort), _stream_handle(stream)), "gee_autotune")
    return tune_table()


def embed_noalloc(edges, Y, K: int, weights=None, *, out=None, stream=None):
    """gee_embed_noalloc: the edge-list embedding with the library's fixed
    scratch array instead of any device allocation (for callers that cannot
    allocate once running).  ``out`` should be preallocated by such callers.
    Calls must not overlap on the GPU."""
    torch = _torch()
    s = _edges_shape(edges)
    n = Y.numel()
    if out is None:
        out = torch.empty((n, K), dtype=torch.float32, device=Y.device)
    rc = lib().gee_embed_noalloc(
        _dev_ptr(edges, torch.int32, "edges"),
        _dev_ptr(weights, torch.float32, "weights", (s,)), s,
        _dev_ptr(Y, torch.int32, "Y", (n,)), n, int(K),
        _dev_ptr(out, torch.float32, "out", (n, K)), _stream_handle(stream))
    check(rc, "gee_embed_noalloc")
    return out


def _host_ptr(a, dtype, name, shape=None):
    import numpy as np
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy {np.dtype(dtype)} array")
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}")
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _host_buf(a):
    """numpy array or pinned CPU tensor -> (pointer, numpy-like view)."""
    try:
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.is_cuda or not a.is_contiguous():
                raise TypeError("host buffers must be contiguous CPU tensors")
            return a.numpy()
    except ImportError:
        pass
    return a


def embed_host(edges, Y, K: int, weights=None, laplacian: bool = False, *,
               strategy="auto", validate_edges: bool = True,
               deterministic: bool = False, out=None, stream=None):
    """gee_embed_host: host (numpy or pinned CPU tensor) inputs and output;
    the library copies them to and from the device."""
    import numpy as np
    edges, Y, weights = _host_buf(edges), _host_buf(Y), _host_buf(weights)
    s = edges.shape[0]
    n = Y.size
    if out is None:
        out = np.empty((n, K), dtype=np.float32)
    outv = _host_buf(out)
    o = options(strategy, validate_edges, deterministic=deterministic)
    rc = lib().gee_embed_host(
        _host_ptr(edges, np.int32, "edges", (s, 2)),
        _host_ptr(weights, np.float32, "weights", (s,)), s,
        _host_ptr(Y, np.int32, "Y", (n,)), n, int(K), int(bool(laplacian)),
        _host_ptr(outv, np.float32, "out", (n, K)), ctypes.byref(o),
        _stream_handle(stream))
    check(rc, "gee_embed_host")
    return out


class Graph:
    """A graph kept resident on the device as a symmetric CSR
    (gee_graph_create); embeds label vectors with gee_embed_graph."""

    def __init__(self, edges, n: int, weights=None, stream=None):
        torch = _torch()
        s = _edges_shape(edges)
        h = ctypes.c_void_p()
        rc = lib().gee_graph_create(
            _dev_ptr(edges, torch.int32, "edges"),
            _dev_ptr(weights, torch.float32, "weights", (s,)), s, int(n),
            _stream_handle(stream), ctypes.byref(h))
        check(rc, "gee_graph_create")
        self._h = h
        self.n = int(n)
        self.s = int(s)
        self.device = edges.device

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("graph is closed")
        return self._h

    def info(self) -> dict:
        vals = [ctypes.c_int64() for _ in range(5)]
        check(lib().gee_graph_info(self.handle, *[ctypes.byref(v) for v in vals]),
              "gee_graph_info")
        return dict(zip(("n", "s", "hub_rows", "hub_arcs", "device_bytes"),
                        (v.value for v in vals)))

    def gathers(self, K: int, stream=None) -> dict:
        """gee_graph_gathers: label gathers of one single-vector pass with K
        classes, by where the label comes from."""
        vals = [ctypes.c_int64() for _ in range(3)]
        check(lib().gee_graph_gathers(self.handle, int(K),
                                      *[ctypes.byref(v) for v in vals],
                                      _stream_handle(stream)), "gee_graph_gathers")
        return dict(zip(("hub_shared", "hub_other", "light"), (v.value for v in vals)))

    def embed(self, Y, K: int, laplacian: bool = False, *, deterministic: bool = False,
              out=None, stream=None):
        """gee_embed_graph; deterministic: float sums in fixed point,
        bitwise reproducible."""
        torch = _torch()
        if out is None:
            out = torch.empty((self.n, K), dtype=torch.float32, device=Y.device)
        o = options(deterministic=deterministic)
        rc = lib().gee_embed_graph(
            self.handle, _dev_ptr(Y, torch.int32, "Y", (self.n,)), int(K),
            int(bool(laplacian)), _dev_ptr(out, torch.float32, "out", (self.n, K)),
            ctypes.byref(o), _stream_handle(stream))
        check(rc, "gee_embed_graph")
        return out

    def embed_multi(self, Y, K: int, laplacian: bool = False, *, deterministic: bool = False,
                    out=None, stream=None):
        """L label vectors (Y: int32 (L, n)) in one pass; returns Z of shape
        (n, L*K) with columns [l*K, (l+1)*K) for vector l
        (gee_embed_graph_multi)."""
        torch = _torch()
        if Y.dim() != 2 or Y.shape[1] != self.n:
            raise ValueError("Y must have shape (L, n)")
        L = Y.shape[0]
        if out is None:
            out = torch.empty((self.n, L * K), dtype=torch.float32, device=Y.device)
        o = options(deterministic=deterministic)
        rc = lib().gee_embed_graph_multi(
            self.handle, _dev_ptr(Y, torch.int32, "Y"), int(L), int(K),
            int(bool(laplacian)), _dev_ptr(out, torch.float32, "out", (self.n, L * K)),
            ctypes.byref(o), _stream_handle(stream))
        check(rc, "gee_embed_graph_multi")
        return out

    def unsupervised(self, Y0, K: int, max_iter: int = 50, *, out=None, stream=None):
        """Unsupervised GEE (gee_unsupervised) from device labels Y0 (every
        label in 0..K-1): returns (labels, Z, rounds, moved per round)."""
        import numpy as np
        torch = _torch()
        Y = Y0.clone()
        if out is None:
            out = torch.empty((self.n, K), dtype=torch.float32, device=Y.device)
        rounds = ctypes.c_int32()
        moved = np.zeros(max(int(max_iter), 1), dtype=np.int64)
        rc = lib().gee_unsupervised(
            self.handle, _dev_ptr(Y, torch.int32, "Y", (self.n,)), int(K), int(max_iter),
            _dev_ptr(out, torch.float32, "out", (self.n, K)), ctypes.byref(rounds),
            ctypes.c_void_p(moved.ctypes.data), _stream_handle(stream))
        check(rc, "gee_unsupervised")
        return Y, out, rounds.value, moved[:rounds.value].tolist()

    def embed_host(self, Y, K: int, laplacian: bool = False, *, deterministic: bool = False,
                   out=None, stream=None):
        import numpy as np
        Yv = _host_buf(Y)
        if out is None:
            out = np.empty((self.n, K), dtype=np.float32)
        outv = _host_buf(out)
        o = options(deterministic=deterministic)
        rc = lib().gee_embed_graph_host(
            self.handle, _host_ptr(Yv, np.int32, "Y", (self.n,)), int(K),
            int(bool(laplacian)), _host_ptr(outv, np.float32, "out", (self.n, K)),
            ctypes.byref(o), _stream_handle(stream))
        check(rc, "gee_embed_graph_host")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gee_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """A gee_server: embedding requests with continuous batching.

    Host arrays (numpy, or numpy views of pinned CPU tensors, which let the
    server overlap copies with other requests' kernels) are referenced until
    ``wait`` returns for their ticket."""

    def __init__(self, hbm_budget_bytes: int = 0, streams: int = 0, max_batch: int = 0,
                 max_batch_edges: int = 0):
        cfg = _lib_mod.ServerConfig()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.streams = int(streams)
        cfg.max_batch = int(max_batch)
        cfg.max_batch_edges = int(max_batch_edges)
        h = ctypes.c_void_p()
        check(lib().gee_server_create(ctypes.byref(cfg), ctypes.byref(h)), "gee_server_create")
        self._h = h
        self._live = {}      # ticket -> (arrays kept alive, Z)
        self._graph_n = {}

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("server is closed")
        return self._h

    def add_graph(self, edges, n: int, weights=None) -> int:
        import numpy as np
        edges = _host_buf(edges)
        weights = _host_buf(weights)
        s = edges.shape[0] if edges.size else 0
        gid = ctypes.c_int64()
        check(lib().gee_server_add_graph(
            self.handle, _host_ptr(edges, np.int32, "edges", (s, 2)),
            _host_ptr(weights, np.float32, "weights", (s,)), s, int(n), ctypes.byref(gid)),
            "gee_server_add_graph")
        self._graph_n[gid.value] = int(n)
        return gid.value

    def drop_graph(self, graph_id: int) -> None:
        check(lib().gee_server_drop_graph(self.handle, int(graph_id)), "gee_server_drop_graph")
        self._graph_n.pop(int(graph_id), None)

    def submit(self, Y, K: int, *, graph=None, edges=None, weights=None,
               laplacian: bool = False, out=None) -> int:
        """Queue one request: a resident graph id (``graph``) or a host edge
        list (``edges`` int32 (s, 2), ``weights``), with labels ``Y``.
        Returns the ticket; ``out`` (float32 (n, K)) receives Z."""
        import numpy as np
        Y = _host_buf(Y)
        n = Y.shape[0]
        if out is None:
            out = np.empty((n, int(K)), dtype=np.float32)
        outv = _host_buf(out)
        r = _lib_mod.Request()
        r.graph = -1 if graph is None else int(graph)
        keep = [Y, out, outv]
        if graph is None:
            edges = _host_buf(edges)
            weights = _host_buf(weights)
            s = edges.shape[0] if edges.size else 0
            r.edges_h = _host_ptr(edges, np.int32, "edges", (s, 2))
            r.weights_h = _host_ptr(weights, np.float32, "weights", (s,))
            r.s = s
            keep += [edges, weights]
        r.n = n
        r.Y_h = _host_ptr(Y, np.int32, "Y", (n,))
        r.K = int(K)
        r.laplacian = int(bool(laplacian))
        r.Z_h = _host_ptr(outv, np.float32, "out", (n, int(K)))
        t = ctypes.c_int64()
        check(lib().gee_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)),
              "gee_server_submit")
        self._live[t.value] = (keep, out)
        return t.value

    def wait(self, ticket: int, raise_on_error: bool = True):
        """Blocks until the request is done: (Z, latency_ms), or with
        ``raise_on_error=False`` (Z, latency_ms, status name)."""
        lat = ctypes.c_double()
        rc = lib().gee_server_wait(self.handle, int(ticket), ctypes.byref(lat))
        _, out = self._live.pop(int(ticket), (None, None))
        if raise_on_error:
            check(rc, "gee_server_wait")
            return out, lat.value
        return out, lat.value, STATUS_NAMES.get(rc, str(rc))

    def cancel(self, ticket: int) -> bool:
        """gee_server_cancel: True if the request was still waiting and is
        now cancelled (its wait then reports GEE_ERR_CANCELLED), False if it
        is already running or done."""
        rc = lib().gee_server_cancel(self.handle, int(ticket))
        return rc == STATUS["GEE_OK"]

    def stats(self) -> dict:
        st = _lib_mod.ServerStats()
        check(lib().gee_server_get_stats(self.handle, ctypes.byref(st)), "gee_server_get_stats")
        return {name: int(getattr(st, name)) for name, _ in st._fields_}

    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().gee_server_destroy(self._h)
        self._h = None
        self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
