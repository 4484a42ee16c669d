"""gee_embed_noalloc, the allocation-free edge-list entry point, through the
C ABI: its output must match gee_embed's on consecutive calls, and both
must match the FP64 oracle.

Callers that cannot allocate device memory once running (a service whose
device memory another allocator divided up at start-up, or code that must
not enter the driver's allocator mid-flight) use this entry point; it keeps
its scratch in a fixed array inside the library.  This file is named to run
last so that a failure here stops a `-x` run only after every other test.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def gee():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_04403_gb300 as gee
    gee.load()
    return gee


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _close(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    nz = want != 0
    assert np.all(got[~nz] == 0)
    if nz.any():
        assert np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz])) <= REL_TOL


def test_matches_gee_embed_on_consecutive_calls(gee):
    """Three calls in a row with different sizes, labels and weights; each
    result equals gee_embed's (bit for bit with unit weights, 1e-5 relative
    with float weights), so nothing left in the shared scratch leaks into
    the next call."""
    cases = []
    n1, s1, K1 = 20000, 300001, 12
    cases.append((graphgen.random_graph(n1, s1, seed=41),
                  graphgen.labels(n1, K1, seed=42, frac_unlabeled=0.2), K1, None))
    n2, s2, K2 = 7001, 90000, 5
    cases.append((graphgen.rmat_edges(13, n2, 0, s2, seed=43),
                  graphgen.labels(n2, K2, seed=44, frac_unlabeled=0.0), K2,
                  graphgen.weights(s2, seed=45)))
    cases.append(cases[0])
    for edges, Y, K, w in cases:
        e_d, y_d = _dev(edges), _dev(Y)
        w_d = None if w is None else _dev(w)
        got = gee.embed_noalloc(e_d, y_d, K, weights=w_d).cpu().numpy()
        want = gee.embed(e_d, y_d, K, weights=w_d).cpu().numpy()
        if w is None:
            assert np.array_equal(got, want)
            assert np.array_equal(got, oracle.embed_counts32(edges, Y, K))
        else:
            _close(got, want)
            _close(got, oracle.embed(edges, Y, K, weights=w))


def test_label_error_is_reported(gee):
    import torch
    edges = graphgen.random_graph(100, 500, seed=1)
    Y = graphgen.labels(100, 3, seed=2).copy()
    Y[7] = 3
    Z = torch.full((100, 3), 2.0, device="cuda")
    with pytest.raises(gee.GeeError) as ei:
        gee.embed_noalloc(_dev(edges), _dev(Y), 3, out=Z)
    assert ei.value.name == "GEE_ERR_LABEL_RANGE"
    assert torch.all(Z == 2.0)
    # a good call right after the failed one
    Y[7] = 1
    got = gee.embed_noalloc(_dev(edges), _dev(Y), 3).cpu().numpy()
    want = gee.embed(_dev(edges), _dev(Y), 3).cpu().numpy()
    assert np.array_equal(got, want)


def test_rejects_more_nodes_than_the_scratch_holds(gee):
    lib = gee.load()
    null = ctypes.c_void_p()
    rc = lib.gee_embed_noalloc(null, null, 0, null, gee.NOALLOC_MAX_NODES + 1, 4,
                               null, null)
    assert gee.STATUS_NAMES[rc] == "GEE_ERR_UNSUPPORTED"
