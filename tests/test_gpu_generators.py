"""The device input generator draws the same values as the host one."""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphgen.build()
    return torch


@pytest.mark.parametrize("scale,n", [(12, 4096), (16, 50000), (26, 65_600_000)])
def test_rmat_device_matches_host(torch, scale, n):
    for start in (0, 123_456_789):
        host = graphgen.rmat_edges(scale, n, start, 20000, seed=3)
        dev = graphgen.rmat_edges_device(scale, n, start, 20000, seed=3).cpu().numpy()
        assert np.array_equal(host, dev)


def test_labels_and_weights_device_match_host(torch):
    for frac in (0.0, 0.1, 1.0):
        h = graphgen.labels(50000, 50, seed=9, frac_unlabeled=frac, start=77)
        d = graphgen.labels_device(50000, 50, seed=9, frac_unlabeled=frac, start=77)
        assert np.array_equal(h, d.cpu().numpy())
    h = graphgen.weights(50000, seed=10, start=5)
    d = graphgen.weights_device(50000, seed=10, start=5)
    assert np.array_equal(h, d.cpu().numpy())


@pytest.mark.parametrize("n,K", [(1000, 1), (12345, 7), (100_000, 32), (2_000_000_000, 3)])
def test_planted_partition_device_matches_host(torch, n, K):
    for start in (0, 987_654_321):
        h = graphgen.planted_edges(n, K, 20000, 10.0, seed=11, start=start)
        d = graphgen.planted_edges_device(n, K, 20000, 10.0, seed=11, start=start)
        assert np.array_equal(h, d.cpu().numpy())
    if n <= 100_000:
        assert np.array_equal(graphgen.planted_labels(n, K),
                              graphgen.planted_labels_device(n, K).cpu().numpy())
