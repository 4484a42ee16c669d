"""The C ABI loads and exports what include/gee.h declares (no GPU needed).

Only host-side logic runs here: symbol lookup, status strings, option
defaults and argument checks that return before any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gee.h")


@pytest.fixture(scope="module")
def gee():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_04403_gb300 as gee
    return gee


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GEE_API\s+[\w\s\*]*?\b(gee_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gee_histogram", "gee_embed", "gee_graph_create",
                     "gee_embed_graph", "gee_graph_destroy", "gee_workspace_bytes",
                     "gee_status_string", "gee_embed_host", "gee_embed_graph_host"):
        assert required in names


def test_library_exports_every_declared_symbol(gee):
    handle = ctypes.CDLL(os.path.join(ROOT, "paper_2402_04403_gb300", "libgee.so"))
    for name in declared_functions():
        assert hasattr(handle, name), f"{name} missing from libgee.so"
    from paper_2402_04403_gb300 import _lib
    assert set(_lib.SIGNATURES) >= set(declared_functions())


def test_generator_and_oracle_libraries_load():
    import graphgen
    import oracle
    g = ctypes.CDLL(graphgen.build())
    for name in ("graphgen_rmat", "graphgen_labels", "graphgen_weights"):
        assert hasattr(g, name)
    o = ctypes.CDLL(oracle.build())
    for name in ("gee_oracle_embed", "gee_oracle_counts", "gee_oracle_embed_rows"):
        assert hasattr(o, name)


def test_status_strings(gee):
    assert gee.status_string(0) == "ok"
    assert "label" in gee.status_string(gee.STATUS["GEE_ERR_LABEL_RANGE"])
    assert gee.status_string(99) == "unknown status"


def test_default_options(gee):
    from paper_2402_04403_gb300 import _lib
    o = _lib.Options()
    _lib.lib().gee_options_default(ctypes.byref(o))
    assert (o.strategy, o.validate_edges, o.private_max_cells, o.block,
            o.deterministic) == (0, 1, 0, 0, 0)


def test_python_options_reach_the_struct(gee):
    o = gee._lib.options("segmented", validate_edges=False, private_max_cells=7,
                         block=64, deterministic=True)
    assert (o.strategy, o.validate_edges, o.private_max_cells, o.block,
            o.deterministic) == (gee.STRATEGIES["segmented"], 0, 7, 64, 1)


def test_fault_hook_and_cancel_need_no_gpu(gee):
    lib = gee.load()
    assert gee.status_string(9) == "request cancelled"
    assert lib.gee_server_cancel(ctypes.c_void_p(), 1) == 1  # no server
    lib.gee_debug_fail_allocs(0)


def test_deterministic_refusals_need_no_gpu(gee):
    """Deterministic float sums need the pull form: the scatter strategies
    and weighted batch problems are refused on the host (GEE_ERR_UNSUPPORTED
    = 8), before any CUDA call."""
    from paper_2402_04403_gb300 import _lib
    lib = gee.load()
    null = ctypes.c_void_p()
    w = ctypes.c_void_p(256)  # a weights pointer that is never read
    for strategy in ("atomic", "private"):
        o = gee._lib.options(strategy, deterministic=True)
        assert lib.gee_embed(null, w, 0, null, 0, 2, 0, null, ctypes.byref(o), null) == 8
        assert lib.gee_embed_host(null, w, 0, null, 0, 2, 0, null, ctypes.byref(o),
                                  null) == 8
    arr = (_lib.Problem * 1)()
    arr[0].weights, arr[0].K = w, 3
    statuses = (ctypes.c_int32 * 1)()
    o = gee._lib.options(deterministic=True)
    assert lib.gee_embed_batch(arr, 1, statuses, ctypes.byref(o), null) == 8
    assert statuses[0] == 8


def test_argument_checks_return_before_any_device_work(gee):
    lib = gee.load()
    null = ctypes.c_void_p()
    # K out of range, negative sizes, bad block: no CUDA call is made
    assert lib.gee_embed(null, null, 0, null, 0, 0, 0, null, None, null) == 1
    assert lib.gee_embed(null, null, 0, null, 0, 256, 0, null, None, null) == 8
    assert lib.gee_embed(null, null, -1, null, 0, 2, 0, null, None, null) == 1
    assert lib.gee_embed(null, null, 5, null, 4, 2, 0, null, None, null) == 1  # NULL edges
    assert lib.gee_histogram(null, 10, 3, null, null) == 1
    assert lib.gee_histogram(null, 0, 0, null, null) == 1
    out = ctypes.c_void_p()
    assert lib.gee_graph_create(null, null, 3, 10, null, ctypes.byref(out)) == 1
    assert lib.gee_embed_graph(null, null, 3, 0, null, None, null) == 1
    lib.gee_graph_destroy(null)  # no-op
    o = gee._lib.options(block=48)
    assert lib.gee_embed(null, null, 0, null, 0, 2, 0, null, ctypes.byref(o), null) == 1


def test_batch_argument_checks_need_no_gpu(gee):
    """gee_embed_batch rejects bad arguments on the host, before any CUDA call."""
    from paper_2402_04403_gb300 import _lib
    lib = gee.load()
    name = lambda rc: gee.STATUS_NAMES[rc]
    assert name(lib.gee_embed_batch(None, -1, None, None, None)) == "GEE_ERR_INVALID_ARG"
    arr = (_lib.Problem * 2)()
    st = (ctypes.c_int * 2)()
    for i in range(2):
        arr[i].K, arr[i].n, arr[i].s = 3, 0, 0
    arr[1].K = 256
    assert name(lib.gee_embed_batch(arr, 2, st, None, None)) == "GEE_ERR_UNSUPPORTED"
    assert name(st[1]) == "GEE_ERR_UNSUPPORTED"
    arr[1].K, arr[1].reserved = 3, 1
    assert name(lib.gee_embed_batch(arr, 2, st, None, None)) == "GEE_ERR_INVALID_ARG"
    arr[1].reserved = 0
    arr[1].s, arr[1].n, arr[1].edges = 4, 10, 4     # 4-byte aligned edge pointer
    arr[1].Y = arr[1].Z = 256
    assert name(lib.gee_embed_batch(arr, 2, st, None, None)) == "GEE_ERR_INVALID_ARG"
    arr[1].edges, arr[1].n = 256, 0                   # edges but no nodes
    assert name(lib.gee_embed_batch(arr, 2, st, None, None)) == "GEE_ERR_NODE_RANGE"


def test_misaligned_edge_lists_are_rejected(gee):
    """Edge lists are read one 8-byte pair at a time; a 4-byte aligned
    pointer is refused before anything runs."""
    lib = gee.load()
    rc = lib.gee_embed(ctypes.c_void_p(4), None, 1, ctypes.c_void_p(256), 2, 2, 0,
                       ctypes.c_void_p(256), None, None)
    assert gee.STATUS_NAMES[rc] == "GEE_ERR_INVALID_ARG"
    g = ctypes.c_void_p()
    rc = lib.gee_graph_create(ctypes.c_void_p(4), None, 1, 2, None, ctypes.byref(g))
    assert gee.STATUS_NAMES[rc] == "GEE_ERR_INVALID_ARG"
    rc = lib.gee_embed_noalloc(ctypes.c_void_p(12), None, 1, ctypes.c_void_p(256), 2, 2,
                               ctypes.c_void_p(256), None)
    assert gee.STATUS_NAMES[rc] == "GEE_ERR_INVALID_ARG"


def test_server_argument_checks_need_no_gpu(gee):
    """The server entry points check their arguments on the host; without a
    CUDA device, creating a server fails with a status instead of crashing."""
    import torch
    from paper_2402_04403_gb300 import _lib
    lib = gee.load()
    name = lambda rc: gee.STATUS_NAMES[rc]
    h = ctypes.c_void_p()
    assert name(lib.gee_server_create(None, None)) == "GEE_ERR_INVALID_ARG"
    cfg = _lib.ServerConfig()
    cfg.streams = 17
    assert name(lib.gee_server_create(ctypes.byref(cfg), ctypes.byref(h))) == "GEE_ERR_INVALID_ARG"
    cfg.streams, cfg.reserved[0] = 0, 1
    assert name(lib.gee_server_create(ctypes.byref(cfg), ctypes.byref(h))) == "GEE_ERR_INVALID_ARG"
    r = _lib.Request()
    t = ctypes.c_int64()
    assert name(lib.gee_server_submit(None, ctypes.byref(r), ctypes.byref(t))) == \
        "GEE_ERR_INVALID_ARG"
    assert name(lib.gee_server_wait(None, 1, None)) == "GEE_ERR_INVALID_ARG"
    assert name(lib.gee_server_drop_graph(None, 0)) == "GEE_ERR_INVALID_ARG"
    lib.gee_server_destroy(None)
    if not torch.cuda.is_available():
        rc = lib.gee_server_create(None, ctypes.byref(h))
        assert rc != 0 and not h.value


def test_tuning_table_drives_auto_without_a_gpu(gee):
    """An installed tuning table decides GEE_AUTO by the nearest grid point
    in (log2 n*K, log2 density); an empty table restores the built-in rule."""
    try:
        gee.tune_set([
            {"log2_cells": 12, "log2_density": 0, "strategy": "segmented", "block": 0},
            {"log2_cells": 20, "log2_density": 0, "strategy": "atomic", "block": 512},
            {"log2_cells": 12, "log2_density": 4, "strategy": "private", "block": 0},
        ])
        assert [c["strategy"] for c in gee.tune_table()] == ["segmented", "atomic", "private"]
        # n*K = 4096 cells, density 1 -> segmented
        assert gee.pick_strategy(2048, 256, 16) == "segmented"
        # n*K = 2^21, density 1 -> nearest is the 2^20 point
        assert gee.pick_strategy(1 << 20, 1 << 17, 16) == "atomic"
        # dense small problem -> private
        assert gee.pick_strategy(32768, 256, 16) == "private"
        # an explicit strategy is not overridden
        assert gee.pick_strategy(2048, 256, 16, strategy="atomic") == "atomic"
        with pytest.raises(gee.GeeError):
            gee.tune_set([{"log2_cells": 1, "log2_density": 0, "strategy": 0}])
    finally:
        gee.tune_set([])
    assert gee.tune_table() == []
    assert gee.pick_strategy(2048, 256, 16) in ("atomic", "private")


def test_missing_library_fails_loudly(gee, monkeypatch, tmp_path):
    """No CPU fallback: without libgee.so every entry point raises."""
    from paper_2402_04403_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libgee.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gee.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gee.status_string(0)


def test_host_tensors_are_refused_not_computed(gee):
    """CPU tensors are rejected before any work: the device entry points
    never compute on the host."""
    import torch
    e = torch.zeros((3, 2), dtype=torch.int32)
    Y = torch.zeros(4, dtype=torch.int32)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gee.embed(e, Y, 2)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gee.Graph(e, 4)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gee.histogram(Y, 2)


def test_product_and_oracle_share_no_code():
    """The library never imports, includes or loads the oracle, and the
    oracle never imports, includes or loads the library."""
    pkg = os.path.join(ROOT, "paper_2402_04403_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                continue
            text = open(os.path.join(dirpath, f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
            assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), f
            assert "gee_oracle" not in text and "libgee_oracle" not in text, f
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if not f.endswith((".py", ".c", ".h")):
            continue
        text = open(os.path.join(odir, f)).read()
        assert "paper_2402_04403_gb300" not in text, f
        assert not re.search(r"#\s*include\s*[<\"](gee\.h|gee_internal)", text), f
        assert "libgee.so" not in text, f
