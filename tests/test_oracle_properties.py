"""Property-based pins of the FP64 oracle (hypothesis draws the graphs):
on any small multigraph -- self-loops, repeated and unlabelled endpoints,
empty classes, signed or non-negative weights -- the oracle equals the dense
closed form (M + M^T) W, and its Laplacian form equals D^-1/2 A D^-1/2 W."""
import numpy as np
import pytest

import oracle
from tests import _pins

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@st.composite
def graphs(draw, signed=True):
    n = draw(st.integers(1, 12))
    K = draw(st.integers(1, 6))
    s = draw(st.integers(0, 40))
    ends = st.integers(0, n - 1)
    edges = np.array(draw(st.lists(st.tuples(ends, ends), min_size=s, max_size=s)),
                     dtype=np.int32).reshape(-1, 2)
    Y = np.array(draw(st.lists(st.integers(-1, K - 1), min_size=n, max_size=n)),
                 dtype=np.int32)
    lo = -4.0 if signed else 0.0
    w = np.array(draw(st.lists(st.floats(lo, 4.0, width=32), min_size=s, max_size=s)),
                 dtype=np.float32) if draw(st.booleans()) else None
    return edges, Y, K, w


@hypothesis.settings(max_examples=300, deadline=None)
@hypothesis.given(graphs())
def test_oracle_is_the_dense_product(g):
    edges, Y, K, w = g
    Z = oracle.embed(edges, Y, K, weights=w)
    Zd = _pins.dense_embedding(edges, Y, K, weights=w)
    scale = 1.0 + np.abs(_pins.dense_embedding(edges, Y, K,
                                               weights=None if w is None else np.abs(w)))
    assert np.all(np.abs(Z - Zd) <= 1e-12 * scale)


@hypothesis.settings(max_examples=300, deadline=None)
@hypothesis.given(graphs(signed=False))
def test_oracle_laplacian_is_the_normalised_product(g):
    edges, Y, K, w = g
    n = Y.size
    A = _pins.dense_adjacency(edges, n, w)
    d = A.sum(axis=1)
    r = np.zeros(n)
    r[d > 0] = 1.0 / np.sqrt(d[d > 0])
    Zd = (r[:, None] * A * r[None, :]) @ _pins.dense_projection(Y, K)
    Z = oracle.embed(edges, Y, K, weights=w, laplacian=True)
    np.testing.assert_allclose(Z, Zd, rtol=1e-12, atol=1e-12)
