"""gee_unsupervised through the C ABI against the oracle's loop: the same
rounds, the same number of nodes moved in every round, the same final
labels bit for bit, and Z the oracle's embedding of those labels."""
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


@pytest.mark.parametrize("n,K,s,ratio,seed", [(20000, 8, 200000, 10.0, 1),
                                               (5000, 3, 30000, 4.0, 2),
                                               (3000, 17, 60000, 30.0, 3)])
def test_planted_partition_matches_oracle_loop(gee, n, K, s, ratio, seed):
    edges = graphgen.planted_edges(n, K, s, ratio, seed=seed)
    Y0 = np.random.default_rng(seed).integers(0, K, n).astype(np.int32)
    want_y, want_rounds, want_moved = oracle.unsupervised(edges, Y0, K, max_iter=40)
    with gee.Graph(_dev(edges), n) as g:
        y, Z, rounds, moved = g.unsupervised(_dev(Y0), K, max_iter=40)
    assert (rounds, moved) == (want_rounds, want_moved)
    assert np.array_equal(y.cpu().numpy(), want_y)
    assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, want_y, K))


def test_rmat_with_hub_rows_and_a_round_limit(gee):
    """Skewed degrees (hub rows in several chunks) and a loop stopped by
    max_iter: the final Z is the embedding of the final labels."""
    n = 30000
    edges = graphgen.rmat_edges(15, n, 0, 400000, seed=8)
    K = 5
    Y0 = graphgen.labels(n, K, seed=9)
    for max_iter in (0, 1, 3):
        want_y, want_rounds, want_moved = oracle.unsupervised(edges, Y0, K, max_iter=max_iter)
        with gee.Graph(_dev(edges), n) as g:
            y, Z, rounds, moved = g.unsupervised(_dev(Y0), K, max_iter=max_iter)
        assert (rounds, moved) == (want_rounds, want_moved)
        assert np.array_equal(y.cpu().numpy(), want_y)
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, want_y, K))


def test_unsupervised_errors(gee):
    n = 500
    edges = graphgen.random_graph(n, 3000, seed=1)
    Y0 = graphgen.labels(n, 4, seed=2)
    with gee.Graph(_dev(edges), n) as g:
        bad = Y0.copy()
        bad[7] = -1
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(bad), 4)
        assert ei.value.name == "GEE_ERR_LABEL_RANGE"
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(Y0), 65)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
    w = graphgen.weights(3000, seed=3)
    with gee.Graph(_dev(edges), n, weights=_dev(w)) as g:
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(Y0), 4)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
