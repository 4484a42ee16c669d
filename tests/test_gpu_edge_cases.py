"""Degenerate inputs through every entry point added around the pass: no
edges, one node, only unknown labels, a star whose hub row spans many
chunks, only self-loops, and the 1,024-column limit with K = 1 -- each
against the oracle."""
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


def _star(n, hub=0, extra=0, seed=0):
    """Every node linked to the hub (a hub row of n-1 arcs, several chunks),
    plus `extra` random edges."""
    leaves = np.arange(n, dtype=np.int32)
    leaves = leaves[leaves != hub]
    e = np.stack([np.full(leaves.size, hub, np.int32), leaves], axis=1)
    if extra:
        e = np.concatenate([e, graphgen.random_graph(n, extra, seed=seed)])
    return e


CASES = {
    "no edges": (np.zeros((0, 2), np.int32), 50),
    "one node, self-loops": (np.zeros((5, 2), np.int32), 1),
    "star, hub in 5 chunks": (_star(10_500, hub=777, extra=3000, seed=3), 10_500),
    "self-loops only": (np.repeat(np.arange(300, dtype=np.int32), 2).reshape(-1, 2), 300),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_resident_single_and_multi(gee, name):
    edges, n = CASES[name]
    with gee.Graph(_dev(edges), n) as g:
        for K, frac in ((3, 0.0), (7, 1.0), (9, 0.3)):
            Y = graphgen.labels(n, K, seed=K, frac_unlabeled=frac)
            want = oracle.embed_counts32(edges, Y, K)
            assert np.array_equal(g.embed(_dev(Y), K).cpu().numpy(), want)
            L = 9  # the lanes-over-vectors form
            Ys = np.stack([graphgen.labels(n, K, seed=100 + l, frac_unlabeled=frac)
                           for l in range(L)])
            Z = g.embed_multi(_dev(Ys), K).cpu().numpy()
            for l in (0, L - 1):
                assert np.array_equal(Z[:, l * K:(l + 1) * K],
                                      oracle.embed_counts32(edges, Ys[l], K)), (K, l)


def test_zero_nodes(gee):
    """n = 0 (no nodes, no edges): every form succeeds with an empty Z, and
    every class size is 0."""
    import torch
    e = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    Y = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert gee.histogram(Y, 4).cpu().tolist() == [0, 0, 0, 0]
    for strategy in ("atomic", "private", "segmented", "binned"):
        for lap in (False, True):
            Z = gee.embed(e, Y, 3, laplacian=lap, strategy=strategy)
            assert tuple(Z.shape) == (0, 3)
    Zh = gee.embed_host(np.zeros((0, 2), np.int32), np.zeros(0, np.int32), 3)
    assert Zh.shape == (0, 3)
    with gee.Graph(e, 0) as g:
        assert g.info()["n"] == 0
        assert tuple(g.embed(Y, 3).shape) == (0, 3)
        assert tuple(g.embed(Y, 3, laplacian=True).shape) == (0, 3)
        Ys = torch.zeros((9, 0), dtype=torch.int32, device="cuda")
        assert tuple(g.embed_multi(Ys, 3).shape) == (0, 27)
        assert g.embed_host(np.zeros(0, np.int32), 3).shape == (0, 3)
    torch.cuda.synchronize()


def test_1024_columns_with_one_class(gee):
    """L = 1,024 label vectors of K = 1 (32 blocks of 32 lanes, odd K)."""
    edges, n = CASES["star, hub in 5 chunks"]
    L, K = 1024, 1
    Ys = np.stack([graphgen.labels(n, K, seed=7 + l, frac_unlabeled=0.5) for l in range(L)])
    with gee.Graph(_dev(edges), n) as g:
        Z = g.embed_multi(_dev(Ys), K).cpu().numpy()
    for l in (0, 31, 32, 1023):
        assert np.array_equal(Z[:, l:l + 1], oracle.embed_counts32(edges, Ys[l], K)), l


def test_batch_and_server_with_degenerate_problems(gee):
    probs = []
    for name in sorted(CASES):
        edges, n = CASES[name]
        for K, frac in ((2, 0.0), (5, 1.0)):
            probs.append((edges, graphgen.labels(n, K, seed=n + K, frac_unlabeled=frac), K))
    Zs = gee.embed_batch([dict(edges=_dev(e), Y=_dev(Y), K=K) for e, Y, K in probs])
    for (e, Y, K), Z in zip(probs, Zs):
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(e, Y, K))
    with gee.Server(streams=2) as srv:
        tickets = [srv.submit(Y, K, edges=e) for e, Y, K in probs]
        edges, n = CASES["no edges"]
        gid = srv.add_graph(edges, n)
        Y = graphgen.labels(n, 4, seed=1)
        tickets.append(srv.submit(Y, 4, graph=gid))
        for (e, Y_, K), t in zip(probs, tickets):
            Z, _ = srv.wait(t)
            assert np.array_equal(Z, oracle.embed_counts32(e, Y_, K))
        Z, _ = srv.wait(tickets[-1])
        assert np.all(Z == 0)


def test_unsupervised_on_degenerate_graphs(gee):
    """No edges, self-loops only, one star hub: every round within the FP32
    rounding slack of the FP64 oracle's round from the same labels (ties
    abound here), Z the embedding of the labels returned."""
    from tests.test_gpu_unsup import _check_choice
    for name in ("no edges", "self-loops only", "star, hub in 5 chunks"):
        edges, n = CASES[name]
        K = min(3, n)
        Y = graphgen.labels(n, K, seed=11)
        with gee.Graph(_dev(edges), n) as g:
            for _ in range(4):
                y, Z, rounds, moved = g.unsupervised(_dev(Y), K, max_iter=1)
                got = y.cpu().numpy()
                _check_choice(edges, Y, K, got)
                assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, got, K)), name
                Y = got


def test_graph_gathers_partition_the_arcs(gee):
    """gee_graph_gathers: the hub rows' arcs split into labels from the
    shared-memory copy and the rest; with the light rows' arcs they are
    every arc (two per edge)."""
    n, s = 300_000, 3_000_000
    edges = graphgen.rmat_edges(19, n, 0, s, seed=12)
    with gee.Graph(_dev(edges), n) as g:
        info, ga, ga64 = g.info(), g.gathers(50), g.gathers(64)
        with pytest.raises(gee.GeeError):
            g.gathers(0)
    for x in (ga, ga64):
        assert x["hub_shared"] + x["hub_other"] == info["hub_arcs"]
        assert x["hub_shared"] + x["hub_other"] + x["light"] == 2 * s
        assert x["hub_shared"] > 0 and x["hub_other"] >= 0
    # below 2^25 nodes the copy holds bytes whatever K
    assert ga == ga64
