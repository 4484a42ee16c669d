"""Error paths of the C ABI on the GPU: statuses, and Z left untouched when
validation fails before the pass."""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gee():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_04403_gb300 as gee
    return gee


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _small():
    n, s, K = 300, 2000, 4
    return graphgen.random_graph(n, s, seed=3), graphgen.labels(n, K, seed=4), n, K


@pytest.mark.parametrize("strategy", ["atomic", "private", "segmented", "binned"])
@pytest.mark.parametrize("bad", [4, -2, 1 << 20])
def test_label_out_of_range_leaves_z(gee, strategy, bad):
    import torch
    edges, Y, n, K = _small()
    Y = Y.copy()
    Y[123] = bad
    Z = torch.full((n, K), 3.5, device="cuda")
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(Y), K, strategy=strategy, out=Z)
    assert ei.value.name == "GEE_ERR_LABEL_RANGE"
    assert torch.all(Z == 3.5)


@pytest.mark.parametrize("strategy", ["atomic", "private", "segmented", "binned"])
@pytest.mark.parametrize("laplacian", [False, True])
def test_node_out_of_range_leaves_z(gee, strategy, laplacian):
    import torch
    edges, Y, n, K = _small()
    edges = edges.copy()
    edges[777, 1] = n
    Z = torch.full((n, K), -1.25, device="cuda")
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(Y), K, strategy=strategy, laplacian=laplacian, out=Z)
    assert ei.value.name == "GEE_ERR_NODE_RANGE"
    assert torch.all(Z == -1.25)
    edges[777, 1] = -5
    with pytest.raises(gee.GeeError):
        gee.embed(_dev(edges), _dev(Y), K, strategy=strategy, laplacian=laplacian, out=Z)
    assert torch.all(Z == -1.25)


def test_node_out_of_range_without_prevalidation(gee):
    import torch
    edges, Y, n, K = _small()
    edges = edges.copy()
    edges[5, 0] = n + 10
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(Y), K, strategy="atomic", validate_edges=False)
    assert ei.value.name == "GEE_ERR_NODE_RANGE"
    torch.cuda.synchronize()  # the bad edge was skipped, the context is fine


def test_graph_rejects_bad_edges(gee):
    edges, Y, n, K = _small()
    edges = edges.copy()
    edges[0, 0] = n
    with pytest.raises(gee.GeeError) as ei:
        gee.Graph(_dev(edges), n)
    assert ei.value.name == "GEE_ERR_NODE_RANGE"


def test_laplacian_rejects_negative_weights(gee):
    edges, Y, n, K = _small()
    w = graphgen.weights(edges.shape[0], seed=1).copy()
    w[10] = -0.5
    for st in ("atomic", "segmented", "binned"):
        with pytest.raises(gee.GeeError) as ei:
            gee.embed(_dev(edges), _dev(Y), K, weights=_dev(w), laplacian=True, strategy=st)
        assert ei.value.name == "GEE_ERR_INVALID_ARG"
    with gee.Graph(_dev(edges), n, weights=_dev(w)) as g:
        g.embed(_dev(Y), K)  # plain weighted embedding is fine
        with pytest.raises(gee.GeeError) as ei:
            g.embed(_dev(Y), K, laplacian=True)
        assert ei.value.name == "GEE_ERR_INVALID_ARG"


def test_bad_scalars(gee):
    edges, Y, n, K = _small()
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(Y), 0)
    assert ei.value.name == "GEE_ERR_INVALID_ARG"
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(Y), 256)
    assert ei.value.name == "GEE_ERR_UNSUPPORTED"


def test_private_falls_back_when_too_large(gee):
    assert gee.pick_strategy(10 ** 6, 10 ** 6, 50, strategy="private") == "atomic"
    assert gee.pick_strategy(10 ** 8, 1000, 5) == "private"
    assert gee.pick_strategy(1000, 10 ** 6, 5) == "atomic"
