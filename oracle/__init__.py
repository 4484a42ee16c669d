"""Serial FP64 CPU oracle for One-Hot Graph Encoder Embedding (Alg. 1 of
"Edge-Parallel Graph Encoder Embedding", arXiv 2402.04403).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg and reference arm are the only callers.  The GPU library never
imports this package and this package never imports the GPU library; they
share no code.

The arithmetic lives in ``gee_oracle.c`` (plain serial C, FP64); this module
builds it with the system C compiler when needed and marshals numpy arrays.
Inputs follow the library's conventions: ``edges`` is an (s, 2) int32 array of
(u, v), ``weights`` an optional float32 array of length s, ``Y`` an int32 array
with classes 0..K-1 and -1 for "class unknown".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gee_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgee_oracle.so")
_LOCK = threading.Lock()
_LIB = None

OK, BAD_ARG, BAD_LABEL, BAD_NODE, NO_MEMORY, BAD_WEIGHT = range(6)
_ERRORS = {
    BAD_ARG: "bad argument",
    BAD_LABEL: "label outside [-1, K)",
    BAD_NODE: "node id outside [0, n)",
    NO_MEMORY: "out of host memory",
    BAD_WEIGHT: "negative weight with the Laplacian variant",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(_ERRORS.get(code, f"oracle error {code}"))
        self.code = code


def build(force: bool = False) -> str:
    """Compile gee_oracle.c into libgee_oracle.so (in place) and return its path."""
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        cc = os.environ.get("CC", "cc")
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([
            cc, "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int32
            ci = ctypes.c_int
            lib.gee_oracle_class_counts.argtypes = [p, i64, i32, p]
            lib.gee_oracle_degrees.argtypes = [p, p, i64, i64, p]
            lib.gee_oracle_embed.argtypes = [p, p, i64, p, i64, i32, ci, p]
            lib.gee_oracle_counts.argtypes = [p, i64, p, i64, i32, p]
            lib.gee_oracle_round_counts.argtypes = [p, i64, i32, p, p]
            lib.gee_oracle_embed_rows.argtypes = [p, p, i64, p, i64, i32, ci,
                                                  p, i64, p, p]
            lib.gee_oracle_set_mutation.argtypes = [ci]
            lib.gee_oracle_unsupervised.argtypes = [p, i64, i64, i32, i32, p, p, p]
            lib.gee_oracle_unsup_round.argtypes = [p, i64, i64, i32, p, p, p, p]
            for f in (lib.gee_oracle_class_counts, lib.gee_oracle_degrees,
                      lib.gee_oracle_embed, lib.gee_oracle_counts,
                      lib.gee_oracle_round_counts, lib.gee_oracle_embed_rows,
                      lib.gee_oracle_unsupervised, lib.gee_oracle_unsup_round):
                f.restype = ci
            lib.gee_oracle_set_mutation.restype = None
            _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _edges(edges):
    e = np.ascontiguousarray(edges, dtype=np.int32)
    if e.ndim != 2 or e.shape[1] != 2:
        e = e.reshape(-1, 2)
    return e


def _weights(weights, s):
    if weights is None:
        return None
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if w.shape != (s,):
        raise ValueError("weights must have one entry per edge")
    return w


def _check(code):
    if code != OK:
        raise OracleError(code)


def set_mutation(code: int) -> None:
    """Plant mistake number ``code`` in the oracle (0 restores it).  Tests only."""
    _lib().gee_oracle_set_mutation(int(code))


def class_counts(Y, K: int) -> np.ndarray:
    """n_k = #{i : Y[i] = k} (Alg. 1, W initialisation)."""
    y = np.ascontiguousarray(Y, dtype=np.int32)
    nk = np.zeros(K, dtype=np.int64)
    _check(_lib().gee_oracle_class_counts(_ptr(y), y.size, K, _ptr(nk)))
    return nk


def degrees(edges, n: int, weights=None) -> np.ndarray:
    """Weighted degree of every node (self-loop counted twice), FP64."""
    e = _edges(edges)
    w = _weights(weights, e.shape[0])
    d = np.zeros(n, dtype=np.float64)
    _check(_lib().gee_oracle_degrees(_ptr(e), _ptr(w), e.shape[0], n, _ptr(d)))
    return d


def embed(edges, Y, K: int, weights=None, laplacian: bool = False) -> np.ndarray:
    """Z = A W of Alg. 1 in FP64, shape (n, K)."""
    e = _edges(edges)
    y = np.ascontiguousarray(Y, dtype=np.int32)
    w = _weights(weights, e.shape[0])
    Z = np.zeros((y.size, K), dtype=np.float64)
    _check(_lib().gee_oracle_embed(_ptr(e), _ptr(w), e.shape[0], _ptr(y),
                                   y.size, K, int(bool(laplacian)), _ptr(Z)))
    return Z


def counts(edges, Y, K: int) -> np.ndarray:
    """Exact unit-weight class counts C (n, K) uint64: Z = C / n_k."""
    e = _edges(edges)
    y = np.ascontiguousarray(Y, dtype=np.int32)
    C = np.zeros((y.size, K), dtype=np.uint64)
    _check(_lib().gee_oracle_counts(_ptr(e), e.shape[0], _ptr(y), y.size, K,
                                    _ptr(C)))
    return C


def round_counts(C, nk) -> np.ndarray:
    """float32 Z with Z[u,k] = RN32(C[u,k] / n_k) (correctly rounded)."""
    c = np.ascontiguousarray(C, dtype=np.uint64)
    nk = np.ascontiguousarray(nk, dtype=np.int64)
    n, K = c.shape
    Z = np.zeros((n, K), dtype=np.float32)
    _check(_lib().gee_oracle_round_counts(_ptr(c), n, K, _ptr(nk), _ptr(Z)))
    return Z


def embed_counts32(edges, Y, K: int) -> np.ndarray:
    """The unit-weight result as the GPU's count path must produce it, bit for
    bit: RN32(C / n_k)."""
    return round_counts(counts(edges, Y, K), class_counts(Y, K))


def embed_rows(edges, Y, K: int, rows, weights=None, laplacian: bool = False,
               with_counts: bool = False):
    """Rows ``rows`` of Z (FP64) and, optionally, their exact integer counts.

    For graphs whose full FP64 Z does not fit in host memory.  ``rows`` is
    sorted and de-duplicated here; the result follows the sorted order, which
    is returned first.
    """
    e = _edges(edges)
    y = np.ascontiguousarray(Y, dtype=np.int32)
    w = _weights(weights, e.shape[0])
    r = np.unique(np.asarray(rows, dtype=np.int64))
    Z = np.zeros((r.size, K), dtype=np.float64)
    C = np.zeros((r.size, K), dtype=np.uint64) if with_counts else None
    _check(_lib().gee_oracle_embed_rows(_ptr(e), _ptr(w), e.shape[0], _ptr(y),
                                        y.size, K, int(bool(laplacian)),
                                        _ptr(r), r.size, _ptr(Z), _ptr(C)))
    return (r, Z, C) if with_counts else (r, Z)


def unsupervised(edges, Y0, K: int, max_iter: int = 50):
    """Unsupervised GEE (gee_oracle_unsupervised): alternate the unit-weight
    embedding with one k-means assignment step from labels Y0 (all known).
    Returns (labels, rounds, moved per round)."""
    e = _edges(edges)
    y = np.array(Y0, dtype=np.int32, copy=True)
    rounds = ctypes.c_int32()
    changes = np.zeros(max(max_iter, 1), dtype=np.int64)
    _check(_lib().gee_oracle_unsupervised(_ptr(e), e.shape[0], y.size, int(K), int(max_iter),
                                          _ptr(y), ctypes.byref(rounds), _ptr(changes)))
    return y, rounds.value, changes[:rounds.value].tolist()


def unsup_round(edges, Y, K: int):
    """One round of the unsupervised loop (gee_oracle_unsup_round) from
    labels Y: returns (next labels, D, T) with D[i, k] the FP64 squared
    distance of node i's embedding to class k's mean (0 for empty classes)
    and T[i, k] = sum_j (|Z[i,j]| + |c[k,j]|)^2, the scale of the rounding
    error a finite-precision evaluation of D[i, k] can carry."""
    e = _edges(edges)
    y = np.ascontiguousarray(Y, dtype=np.int32)
    nxt = np.zeros(max(y.size, 1), dtype=np.int32)
    D = np.zeros((y.size, K), dtype=np.float64)
    T = np.zeros((y.size, K), dtype=np.float64)
    _check(_lib().gee_oracle_unsup_round(_ptr(e), e.shape[0], y.size, int(K), _ptr(y),
                                         _ptr(nxt), _ptr(D), _ptr(T)))
    return nxt[:y.size], D, T
