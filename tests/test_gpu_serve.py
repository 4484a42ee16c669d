"""The serving runtime (gee_server_*) through the C ABI: requests submitted
in a burst or from several client threads are batched and overlapped, and
every result is the same as that request's solo call (bit for bit with
unit weights, 1e-5 relative with float weights); admission respects the
memory budget; a failing request does not disturb the others."""
import threading

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


def _close(got, want, what):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    nz = want != 0
    assert np.all(got[~nz] == 0), what
    if nz.any():
        rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        assert rel.max() <= REL_TOL, f"{what}: {rel.max():.3e}"


@pytest.fixture(scope="module")
def graphs():
    """Two graphs to keep resident: weighted R-MAT with multi-chunk hub rows,
    unweighted planted partition."""
    nA, sA = 20000, 300000
    eA = graphgen.rmat_edges(15, nA, 0, sA, seed=71)
    wA = graphgen.weights(sA, seed=72)
    nB, sB = 30000, 200000
    eB = graphgen.planted_edges(nB, 6, sB, 10.0, seed=73)
    return (eA, wA, nA), (eB, None, nB)


def _edge_requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(50, 20000))
        K = int(rng.integers(2, 40))
        s = int(n * rng.uniform(1, 20))
        e = graphgen.planted_edges(n, min(K, n), s, 10.0, seed=seed * 100 + i)
        Y = graphgen.labels(n, K, seed=seed * 100 + i, frac_unlabeled=0.1)
        w = graphgen.weights(s, seed=seed * 100 + i) if i % 2 else None
        out.append((e, w, Y, K))
    return out


def test_mixed_burst_equals_solo_calls(gee, graphs):
    (eA, wA, nA), (eB, _, nB) = graphs
    with gee.Server(streams=4, max_batch=64) as srv:
        gA = srv.add_graph(eA, nA, weights=wA)
        gB = srv.add_graph(eB, nB)
        reqs = []
        for e, w, Y, K in _edge_requests(24, seed=1):
            reqs.append(("edges", (e, w, Y, K), srv.submit(Y, K, edges=e, weights=w)))
        for l in range(12):   # same graph and K: one multi-label group (wide form)
            Y = graphgen.labels(nB, 9, seed=500 + l, frac_unlabeled=0.05)
            reqs.append(("B", (Y, 9, False), srv.submit(Y, 9, graph=gB)))
        for l in range(3):    # a small group of weighted re-labelings
            Y = graphgen.labels(nA, 5, seed=600 + l, frac_unlabeled=0.1)
            reqs.append(("A", (Y, 5, False), srv.submit(Y, 5, graph=gA)))
        Y = graphgen.labels(nA, 7, seed=700)
        reqs.append(("A", (Y, 7, True), srv.submit(Y, 7, graph=gA, laplacian=True)))
        results = [(kind, args, srv.wait(t)) for kind, args, t in reqs]
        st = srv.stats()
    assert st["completed"] == st["submitted"] == len(reqs) and st["failed"] == 0
    assert st["groups"] < len(reqs) and st["max_group"] >= 12
    assert st["graph_launches"] >= 1  # edge-list groups ran as CUDA graphs
    with gee.Graph(_dev(eA), nA, weights=_dev(wA)) as GA, gee.Graph(_dev(eB), nB) as GB:
        for kind, args, (Z, lat) in results:
            assert lat > 0
            if kind == "edges":
                e, w, Y, K = args
                if w is None:
                    assert np.array_equal(Z, oracle.embed_counts32(e, Y, K))
                else:
                    _close(Z, oracle.embed(e, Y, K, weights=w), "edge-list request vs oracle")
                    solo = gee.embed(_dev(e), _dev(Y), K, weights=_dev(w)).cpu().numpy()
                    _close(Z, solo, "edge-list request vs its solo call")
            else:
                Y, K, lap = args
                g = GA if kind == "A" else GB
                solo = g.embed(_dev(Y), K, laplacian=lap).cpu().numpy()
                if kind == "B":
                    assert np.array_equal(Z, solo)
                    assert np.array_equal(Z, oracle.embed_counts32(eB, Y, K))
                else:
                    _close(Z, oracle.embed(eA, Y, K, weights=wA, laplacian=lap),
                           f"re-label {kind} lap={lap} vs oracle")
                    _close(Z, solo, f"re-label {kind} lap={lap} vs its solo call")
    # spot checks against the oracle itself
    Y, K, _ = results[24][1]
    assert np.array_equal(results[24][2][0], oracle.embed_counts32(eB, Y, K))


def test_concurrent_clients(gee, graphs):
    (eB, _, nB) = graphs[1]
    errors = []
    with gee.Server(streams=3, max_batch=16) as srv:
        gB = srv.add_graph(eB, nB)

        def client(cid):
            rng = np.random.default_rng(cid)
            try:
                for j in range(12):
                    if j % 3 == 0:
                        Y = graphgen.labels(nB, 4, seed=cid * 1000 + j)
                        Z, _ = srv.wait(srv.submit(Y, 4, graph=gB))
                        want = oracle.embed_counts32(eB, Y, 4)
                    else:
                        n = int(rng.integers(10, 3000))
                        e = graphgen.random_graph(n, 4 * n, seed=cid * 1000 + j)
                        Y = graphgen.labels(n, 6, seed=cid * 1000 + j, frac_unlabeled=0.2)
                        Z, _ = srv.wait(srv.submit(Y, 6, edges=e))
                        want = oracle.embed_counts32(e, Y, 6)
                    if not np.array_equal(Z, want):
                        errors.append((cid, j))
            except Exception as exc:  # reported below
                errors.append((cid, repr(exc)))

        threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert srv.stats()["completed"] == 48
    assert not errors, errors


def test_admission_by_budget(gee):
    """With a budget that holds about one request at a time everything still
    completes, in-flight bytes stay under the budget, and a request larger
    than the whole budget fails with GEE_ERR_OOM."""
    reqs = _edge_requests(10, seed=3)
    biggest = max(e.shape[0] * 12 + Y.size * (8 + 4 * K) for e, w, Y, K in reqs)
    budget = 2 * biggest + (1 << 20)
    with gee.Server(hbm_budget_bytes=budget, streams=4) as srv:
        tickets = [srv.submit(Y, K, edges=e, weights=w) for e, w, Y, K in reqs]
        n = 200_000
        e = graphgen.random_graph(n, budget // 8, seed=9)
        Y = graphgen.labels(n, 3, seed=9)
        big = srv.submit(Y, 3, edges=e)
        for (e_, w, Y_, K), t in zip(reqs, tickets):
            Z, _ = srv.wait(t)
            if w is None:
                assert np.array_equal(Z, oracle.embed_counts32(e_, Y_, K))
        _, _, status = srv.wait(big, raise_on_error=False)
        assert status == "GEE_ERR_OOM"
        st = srv.stats()
        assert 0 < st["peak_inflight_bytes"] <= budget


def test_bad_label_fails_only_its_request(gee, graphs):
    (eB, _, nB) = graphs[1]
    with gee.Server(streams=1) as srv:
        gB = srv.add_graph(eB, nB)
        # hold the only slot so the re-labelings queue up and group
        e = graphgen.random_graph(50000, 2_000_000, seed=1)
        Yb = graphgen.labels(50000, 3, seed=1)
        first = srv.submit(Yb, 3, edges=e)
        Ys = [graphgen.labels(nB, 5, seed=800 + l) for l in range(6)]
        Ys[3][123] = 5
        tickets = [srv.submit(Y, 5, graph=gB) for Y in Ys]
        srv.wait(first)
        out = [srv.wait(t, raise_on_error=False) for t in tickets]
        assert [o[2] for o in out] == ["GEE_OK"] * 3 + ["GEE_ERR_LABEL_RANGE"] + ["GEE_OK"] * 2
        for l in (0, 5):
            assert np.array_equal(out[l][0], oracle.embed_counts32(eB, Ys[l], 5))
        # a graph with queued work cannot be dropped; afterwards it can
        # (the edge list ahead of it keeps the re-labeling queued)
        ahead = srv.submit(Yb, 3, edges=e)
        t = srv.submit(Ys[0], 5, graph=gB)
        with pytest.raises(gee.GeeError):
            srv.drop_graph(gB)
        srv.wait(ahead)
        srv.wait(t)
        srv.drop_graph(gB)
        with pytest.raises(gee.GeeError):
            srv.submit(Ys[0], 5, graph=gB)


def test_multi_group_outputs_page_locked_and_pageable(gee, graphs):
    """A fused multi-label group returns each vector's columns to that
    request's own output: page-locked outputs (placed so that no two start at
    the same offset within a 128-byte line) are written over the host link by
    the split kernel, a pageable one by a strided copy.  Every output equals
    the oracle and no float around the outputs changes."""
    import torch
    (eB, _, nB) = graphs[1]
    cases = ((9, 12), (5, 3), (64, 16))  # (K, L): wide and narrow forms; 16 x 64 = 1,024
    with gee.Server(streams=1) as srv:
        gB = srv.add_graph(eB, nB)
        # hold the only slot so the re-labelings queue up and group
        e = graphgen.random_graph(50000, 2_000_000, seed=2)
        Yb = graphgen.labels(50000, 3, seed=2)
        for K, L in cases:
            Ys = [graphgen.labels(nB, K, seed=900 + 37 * K + l, frac_unlabeled=0.1)
                  for l in range(L)]
            gaps = [1 + 7 * l for l in range(L)]  # floats before each output
            total = sum(gaps) + L * nB * K + 32
            buf = torch.full((total,), float("nan"), dtype=torch.float32, pin_memory=True)
            flat = buf.numpy()
            outs, spans, pos = [], [], 0
            for l in range(L):
                pos += gaps[l]
                if l == 1:
                    outs.append(np.empty((nB, K), np.float32))  # pageable
                else:
                    outs.append(flat[pos:pos + nB * K].reshape(nB, K))
                    spans.append((pos, pos + nB * K))
                pos += nB * K
            first = srv.submit(Yb, 3, edges=e)
            tickets = [srv.submit(Y, K, graph=gB, out=o) for Y, o in zip(Ys, outs)]
            srv.wait(first)
            for l, (Y, t) in enumerate(zip(Ys, tickets)):
                srv.wait(t)
                assert np.array_equal(outs[l], oracle.embed_counts32(eB, Y, K)), (K, L, l)
            outside = np.ones(total, bool)
            for a, b in spans:
                outside[a:b] = False
            assert np.all(np.isnan(flat[outside])), (K, L)
        assert srv.stats()["max_group"] == 16


def test_requests_overlap_on_the_device(gee):
    """Continuous batching, not a queue: four requests submitted together,
    one group each on four slots, finish in well under four times one
    request's time alone -- one request's copies over the host link run
    while another's kernels run -- the server saw several groups in flight,
    and every result equals the oracle (sampled rows)."""
    import time
    import torch
    n, s, K = 1_000_000, 12_000_000, 16
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    # page-locked buffers, as a serving client's are (a copy from pageable
    # memory holds the calling thread, here the scheduler)
    e = pin(graphgen.rmat_edges(20, n, 0, s, seed=31))
    Y = pin(graphgen.labels(n, K, seed=32, frac_unlabeled=0.1))
    outs = [torch.empty((n, K), dtype=torch.float32).pin_memory().numpy() for _ in range(4)]
    with gee.Server(streams=4, max_batch=1) as srv:
        srv.wait(srv.submit(Y, K, edges=e, out=outs[0]))  # warm-up
        t = time.perf_counter()
        srv.wait(srv.submit(Y, K, edges=e, out=outs[0]))
        alone = time.perf_counter() - t
        t = time.perf_counter()
        tickets = [srv.submit(Y, K, edges=e, out=o) for o in outs]
        for tk in tickets:
            srv.wait(tk)
        together = time.perf_counter() - t
        st = srv.stats()
    print(f"one request {1e3 * alone:.2f} ms, four at once {1e3 * together:.2f} ms")
    assert st["max_concurrent"] >= 2
    assert together < 0.9 * 4 * alone
    rows = np.random.default_rng(36).integers(0, n, 2000)
    r, _, C = oracle.embed_rows(e, Y, K, rows, with_counts=True)
    want = oracle.round_counts(C, oracle.class_counts(Y, K))
    for o in outs:
        assert np.array_equal(o[r], want)


def test_max_concurrent_counts_groups_in_flight(gee, graphs):
    """A burst of independent edge-list requests larger than one group
    (max_batch = 2) on four slots keeps more than one group on the GPU."""
    reqs = _edge_requests(16, seed=7)
    with gee.Server(streams=4, max_batch=2) as srv:
        tickets = [srv.submit(Y, K, edges=e, weights=w) for e, w, Y, K in reqs]
        outs = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert st["groups"] >= 8 and st["max_concurrent"] >= 2
    for (e, w, Y, K), Z in zip(reqs, outs):
        if w is None:
            assert np.array_equal(Z, oracle.embed_counts32(e, Y, K))
        else:
            _close(Z, oracle.embed(e, Y, K, weights=w), "burst request vs oracle")
