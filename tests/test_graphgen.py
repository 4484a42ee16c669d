"""Host-side checks of the seeded input generators."""
import numpy as np
import pytest

import graphgen


# Known-answer vectors of Philox4x32-10 published with the Random123 library
# (Salmon et al., SC'11): (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2,
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(ctr, key, out):
    got = graphgen.philox4x32_10(*[[c] for c in ctr], *key)
    assert tuple(int(x[0]) for x in got) == out


def test_rmat_is_seeded_and_sliceable():
    a = graphgen.rmat_edges(12, 4000, 0, 5000, seed=9)
    b = graphgen.rmat_edges(12, 4000, 1000, 2000, seed=9)
    assert np.array_equal(a[1000:3000], b)
    c = graphgen.rmat_edges(12, 4000, 0, 5000, seed=10)
    assert not np.array_equal(a, c)
    assert a.min() >= 0 and a.max() < 4000


def test_rmat_quadrant_frequencies():
    """Without the id bijection R-MAT's first level is quadrant a/b/c/d with
    probabilities 0.57/0.19/0.19/0.05; the bijection preserves the degree
    multiset, so check the skew through the degree distribution instead:
    the top 1% of nodes must carry far more than 1% of endpoints."""
    e = graphgen.rmat_edges(16, 1 << 16, 0, 1 << 20, seed=3)
    deg = np.bincount(e.ravel(), minlength=1 << 16)
    top = np.sort(deg)[::-1][: (1 << 16) // 100].sum() / deg.sum()
    assert top > 0.15


def test_rmat_thresholds():
    assert graphgen.rmat_thresholds(0.57, 0.19, 0.19) == (37356, 49807, 62259)


def test_permutation_is_bijective():
    for scale in (1, 5, 10, 13):
        x = np.arange(1 << scale, dtype=np.uint64)
        y = graphgen.permute_ids(x, scale, seed=77)
        assert np.array_equal(np.sort(y), x)


def test_labels_and_weights():
    y = graphgen.labels(200000, 50, seed=4, frac_unlabeled=0.1)
    assert y.min() == -1 and y.max() == 49
    assert abs((y == -1).mean() - 0.1) < 0.005
    counts = np.bincount(y[y >= 0], minlength=50)
    assert counts.min() > 0.9 * counts.mean()
    w = graphgen.weights(100000, seed=5)
    assert w.dtype == np.float32 and w.min() > 0 and w.max() <= 1.0
    assert abs(w.mean() - 0.5) < 0.01


def test_sbm_structure(tiny_sbm_graph):
    e, y = tiny_sbm_graph
    assert y.size == 10000 and set(np.unique(y)) == set(range(5))
    assert np.all(e[:, 0] != e[:, 1])
    same = y[e[:, 0]] == y[e[:, 1]]
    # expected within-block share: 5*C(2000,2)*0.02 / 279,900
    assert abs(same.mean() - 199900 / 279900) < 0.01
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = lo.astype(np.int64) * 10000 + hi
    assert np.unique(key).size == key.size  # simple graph


def test_planted_partition_structure():
    """Blocks are floor(i K / n) (sizes differ by at most one); endpoints are
    in range; the share of edges inside a block matches its threshold and the
    share p_in (b-1) / (p_in (b-1) + p_out (n-b)) of an SBM node's expected
    edges; K = 1 keeps every edge inside the single block."""
    n, K, s = 10007, 9, 300000
    y = graphgen.planted_labels(n, K)
    sizes = np.bincount(y)
    assert sizes.size == K and sizes.max() - sizes.min() <= 1
    assert np.array_equal(graphgen.planted_block_start(np.arange(K + 1), n, K),
                          np.concatenate([[0], np.cumsum(sizes)]))
    e = graphgen.planted_edges(n, K, s, 10.0, seed=4)
    assert e.min() >= 0 and e.max() < n
    same = (y[e[:, 0]] == y[e[:, 1]]).mean()
    b = n / K
    q = 10 * (b - 1) / (10 * (b - 1) + n - b)
    assert abs(same - q) < 4 * np.sqrt(q * (1 - q) / s)
    assert abs(graphgen.planted_same_threshold(n, K, 10.0) / 2**32 - q) < 1e-9
    # first endpoints are uniform over nodes: each block gets its share
    frac = np.bincount(y[e[:, 0]], minlength=K) / s
    assert np.allclose(frac, sizes / n, atol=0.01)
    e1 = graphgen.planted_edges(500, 1, 1000, 10.0, seed=4)
    assert e1.min() >= 0 and e1.max() < 500
    # same seed, sliced: identical edges
    assert np.array_equal(graphgen.planted_edges(n, K, 100, 10.0, seed=4, start=50),
                          e[50:150])


def test_host_batching_does_not_change_values(monkeypatch):
    """The host generators draw in batches; any batch size gives the same
    edges, labels and weights (each value is a function of its index)."""
    ref = (graphgen.rmat_edges(12, 3000, 5, 1000, seed=8),
           graphgen.labels(1000, 7, seed=9, frac_unlabeled=0.3, start=11),
           graphgen.weights(1000, seed=10, start=13))
    monkeypatch.setattr(graphgen, "_HOST_CHUNK", 7)
    got = (graphgen.rmat_edges(12, 3000, 5, 1000, seed=8),
           graphgen.labels(1000, 7, seed=9, frac_unlabeled=0.3, start=11),
           graphgen.weights(1000, seed=10, start=13))
    for a, b in zip(ref, got):
        assert a.dtype == b.dtype and np.array_equal(a, b)
