"""ctypes declarations of libgee.so (include/gee.h).  Argument marshalling
only; every step of the embedding runs in the library's CUDA kernels.  There
is no fallback: if the library is missing, loading fails with an error."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgee.so")

STATUS_NAMES = {
    0: "GEE_OK",
    1: "GEE_ERR_INVALID_ARG",
    2: "GEE_ERR_LABEL_RANGE",
    3: "GEE_ERR_NODE_RANGE",
    4: "GEE_ERR_OVERFLOW",
    5: "GEE_ERR_OOM",
    6: "GEE_ERR_CUDA",
    7: "GEE_ERR_TIMEOUT",
    8: "GEE_ERR_UNSUPPORTED",
    9: "GEE_ERR_CANCELLED",
}
STATUS = {v: k for k, v in STATUS_NAMES.items()}
STRATEGIES = {"auto": 0, "atomic": 1, "private": 2, "segmented": 3, "binned": 4}
STRATEGY_NAMES = {v: k for k, v in STRATEGIES.items()}
MAX_CLASSES = 255
MAX_COLUMNS = 1024
NOALLOC_MAX_NODES = (16 << 20) - 2048
HUB_DEGREE = 128


class GeeError(RuntimeError):
    """A libgee call returned a status other than GEE_OK."""

    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        self.name = STATUS_NAMES.get(self.code, f"status {code}")
        msg = f"{what}: {self.name}" if what else self.name
        super().__init__(msg)


class Options(ctypes.Structure):
    _fields_ = [
        ("strategy", ctypes.c_int32),
        ("validate_edges", ctypes.c_int32),
        ("private_max_cells", ctypes.c_int64),
        ("block", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
    ]


class KernelTime(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_int64),
        ("total_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double),
    ]


class Problem(ctypes.Structure):
    """gee_problem: one problem of gee_embed_batch."""
    _fields_ = [
        ("edges", ctypes.c_void_p),
        ("weights", ctypes.c_void_p),
        ("s", ctypes.c_int64),
        ("Y", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("K", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("Z", ctypes.c_void_p),
    ]


class TuneCell(ctypes.Structure):
    """gee_tune_cell: one grid point of the GEE_AUTO tuning table."""
    _fields_ = [
        ("log2_cells", ctypes.c_int32),
        ("log2_density", ctypes.c_int32),
        ("strategy", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("ms_atomic", ctypes.c_float),
        ("ms_private", ctypes.c_float),
        ("ms_segmented", ctypes.c_float),
        ("reserved", ctypes.c_float),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_int64),
        ("streams", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("max_batch_edges", ctypes.c_int64),
        ("reserved", ctypes.c_int64 * 2),
    ]


class Request(ctypes.Structure):
    """gee_request: one request to a gee_server."""
    _fields_ = [
        ("graph", ctypes.c_int64),
        ("edges_h", ctypes.c_void_p),
        ("weights_h", ctypes.c_void_p),
        ("s", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("Y_h", ctypes.c_void_p),
        ("K", ctypes.c_int32),
        ("laplacian", ctypes.c_int32),
        ("Z_h", ctypes.c_void_p),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "submitted", "completed", "failed", "groups", "batched_requests", "max_group",
        "max_concurrent", "resident_bytes", "peak_inflight_bytes", "graph_launches")]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_OPT = ctypes.POINTER(Options)
SIGNATURES = {
    "gee_options_default": (None, [_OPT]),
    "gee_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gee_histogram": (ctypes.c_int, [_P, _I64, _I32, _P, _P]),
    "gee_embed": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _I32, _I32, _P, _OPT, _P]),
    "gee_embed_host": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _I32, _I32, _P, _OPT, _P]),
    "gee_graph_create": (ctypes.c_int, [_P, _P, _I64, _I64, _P, ctypes.POINTER(_P)]),
    "gee_embed_graph": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _OPT, _P]),
    "gee_embed_graph_host": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _OPT, _P]),
    "gee_embed_graph_multi": (ctypes.c_int, [_P, _P, _I32, _I32, _I32, _P, _OPT, _P]),
    "gee_graph_info": (ctypes.c_int, [_P] + [ctypes.POINTER(_I64)] * 5),
    "gee_graph_gathers": (ctypes.c_int, [_P, _I32] + [ctypes.POINTER(_I64)] * 3 + [_P]),
    "gee_graph_destroy": (None, [_P]),
    "gee_pick_strategy": (ctypes.c_int, [_I64, _I64, _I32, _OPT]),
    "gee_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I32, _I32, _I32, _OPT]),
    "gee_embed_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _I32, _P, _P]),
    "gee_embed_batch": (ctypes.c_int, [ctypes.POINTER(Problem), _I32,
                                       ctypes.POINTER(ctypes.c_int), _OPT, _P]),
    "gee_unsupervised": (ctypes.c_int, [_P, _P, _I32, _I32, _P, ctypes.POINTER(_I32),
                                        _P, _P]),
    "gee_autotune": (ctypes.c_int, [_I32, _P]),
    "gee_tune_get": (_I32, [ctypes.POINTER(TuneCell), _I32]),
    "gee_tune_set": (ctypes.c_int, [ctypes.POINTER(TuneCell), _I32]),
    "gee_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    "gee_server_add_graph": (ctypes.c_int, [_P, _P, _P, _I64, _I64, ctypes.POINTER(_I64)]),
    "gee_server_drop_graph": (ctypes.c_int, [_P, _I64]),
    "gee_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(_I64)]),
    "gee_server_wait": (ctypes.c_int, [_P, _I64, ctypes.POINTER(ctypes.c_double)]),
    "gee_server_cancel": (ctypes.c_int, [_P, _I64]),
    "gee_debug_fail_allocs": (None, [_I32]),
    "gee_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "gee_server_destroy": (None, [_P]),
    "gee_profile_enable": (None, [_I32]),
    "gee_profile_read": (_I32, [ctypes.POINTER(KernelTime), _I32]),
}


def lib():
    """The loaded libgee.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` "
                    "(there is no CPU fallback)")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(code: int, what: str = "") -> None:
    if code != 0:
        raise GeeError(code, what)


def options(strategy="auto", validate_edges=True, private_max_cells=0, block=0,
            deterministic=False):
    o = Options()
    lib().gee_options_default(ctypes.byref(o))
    o.strategy = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
    o.validate_edges = 1 if validate_edges else 0
    o.private_max_cells = int(private_max_cells)
    o.block = int(block)
    o.deterministic = 1 if deterministic else 0
    return o
