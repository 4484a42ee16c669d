"""Failure handling without a GPU fault: allocation failures injected on
the host (gee_debug_fail_allocs) make the calls that meet them return
GEE_ERR_OOM and leave the library usable, and server requests cancelled
before admission finish with GEE_ERR_CANCELLED while the others complete
as usual."""
import time

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


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


def test_injected_allocation_failures(gee):
    n, K = 5000, 6
    e = graphgen.random_graph(n, 40000, seed=3)
    Y = graphgen.labels(n, K, seed=4, frac_unlabeled=0.1)
    want = oracle.embed_counts32(e, Y, K)
    try:
        for strategy in ("atomic", "segmented", "binned"):
            gee.debug_fail_allocs(1)
            with pytest.raises(gee.GeeError) as ei:
                gee.embed(_dev(e), _dev(Y), K, strategy=strategy)
            assert ei.value.name == "GEE_ERR_OOM", strategy
            gee.debug_fail_allocs(0)
            assert np.array_equal(gee.embed(_dev(e), _dev(Y), K, strategy=strategy)
                                  .cpu().numpy(), want), strategy
        gee.debug_fail_allocs(1)  # graph creation: its first array fails
        with pytest.raises(gee.GeeError) as ei:
            gee.Graph(_dev(e), n)
        assert ei.value.name == "GEE_ERR_OOM"
        gee.debug_fail_allocs(0)
        with gee.Graph(_dev(e), n) as g:
            gee.debug_fail_allocs(1)
            with pytest.raises(gee.GeeError) as ei:
                g.embed(_dev(Y), K)
            assert ei.value.name == "GEE_ERR_OOM"
            gee.debug_fail_allocs(0)
            assert np.array_equal(g.embed(_dev(Y), K).cpu().numpy(), want)
    finally:
        gee.debug_fail_allocs(0)


def test_cancel_waiting_requests(gee):
    nB, KB = 30000, 5
    eB = graphgen.planted_edges(nB, 6, 200000, 10.0, seed=73)
    # every input made before the first submission, so the queue fills
    # faster than the first request (a 1.28 GB Z to return) can finish
    n_big = 5_000_000
    e_big = graphgen.random_graph(n_big, 10_000_000, seed=1)
    Y_big = graphgen.labels(n_big, 64, seed=1)
    small = []
    for i in range(6):
        n = 2000 + 100 * i
        small.append((graphgen.random_graph(n, 8 * n, seed=10 + i),
                      graphgen.labels(n, 4, seed=20 + i)))
    Yr = graphgen.labels(nB, KB, seed=30)
    with gee.Server(streams=1) as srv:
        gB = srv.add_graph(eB, nB)
        first = srv.submit(Y_big, 64, edges=e_big)
        deadline = time.time() + 30
        while srv.stats()["groups"] < 1 and time.time() < deadline:
            time.sleep(0.0002)  # admitted alone: later edge lists wait
        tickets = [srv.submit(Y, 4, edges=e) for e, Y in small]
        relabel = srv.submit(Yr, KB, graph=gB)
        cancelled = {i for i in (1, 3, 5) if srv.cancel(tickets[i])}
        relabel_cancelled = srv.cancel(relabel)
        srv.wait(first)
        for i, ((e, Y), t) in enumerate(zip(small, tickets)):
            Z, _, status = srv.wait(t, raise_on_error=False)
            if i in cancelled:
                assert status == "GEE_ERR_CANCELLED", i
            else:
                assert status == "GEE_OK", i
                assert np.array_equal(Z, oracle.embed_counts32(e, Y, 4)), i
        _, _, status = srv.wait(relabel, raise_on_error=False)
        assert status == ("GEE_ERR_CANCELLED" if relabel_cancelled else "GEE_OK")
        assert cancelled == {1, 3, 5} and relabel_cancelled  # the slot was held
        # a done request cannot be cancelled; the graph has no users left
        t = srv.submit(Yr, KB, graph=gB)
        srv.wait(t)
        assert not srv.cancel(t)
        srv.drop_graph(gB)
        st = srv.stats()
        assert st["completed"] == st["submitted"]
