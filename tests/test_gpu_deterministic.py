"""The deterministic option (gee_options.deterministic): float sums in
64-bit fixed point, so weighted and Laplacian results are the same bits on
every call, on graphs built from the edge list in any order, in the host
and multi-label forms and in the SEGMENTED edge-list call -- and within an
ulp or so of the FP64 oracle (arc values are rounded to units of 2^-S with
S about 48 here, then each cell is divided once in FP64).  The forms that
add floats with global atomics refuse the option."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

ULPS = 2.4e-7  # two float ulps, relative


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


@pytest.fixture(scope="module")
def weighted_rmat():
    """R-MAT scale 16 with float weights (hub rows of many chunks), and the
    same edges in another order."""
    n = 1 << 16
    edges = graphgen.rmat_edges(16, n, 0, 1 << 20, seed=61)
    w = graphgen.weights(edges.shape[0], seed=62)
    perm = np.random.default_rng(63).permutation(edges.shape[0])
    return n, edges, w, edges[perm], w[perm]


def _close_to_oracle(Z, z64):
    nz = z64 != 0
    assert np.all(Z[~nz] == 0)
    rel = np.abs(Z[nz].astype(np.float64) - z64[nz]) / np.abs(z64[nz])
    assert rel.max() <= ULPS, rel.max()


@pytest.mark.parametrize("K,lap", [(5, False), (50, False), (7, True)])
def test_bitwise_across_calls_and_edge_orders(gee, weighted_rmat, K, lap):
    import torch
    n, e, w, e2, w2 = weighted_rmat
    Y = graphgen.labels(n, K, seed=64 + K, frac_unlabeled=0.1)
    with gee.Graph(_dev(e), n, weights=_dev(w)) as A, \
            gee.Graph(_dev(e2), n, weights=_dev(w2)) as B:
        za = A.embed(_dev(Y), K, laplacian=lap, deterministic=True).cpu().numpy()
        za2 = A.embed(_dev(Y), K, laplacian=lap, deterministic=True).cpu().numpy()
        zb = B.embed(_dev(Y), K, laplacian=lap, deterministic=True).cpu().numpy()
        Zp = torch.empty((n, K), dtype=torch.float32).pin_memory()
        A.embed_host(torch.from_numpy(Y).pin_memory(), K, laplacian=lap,
                     deterministic=True, out=Zp)
    assert np.array_equal(za, za2)
    assert np.array_equal(za, zb)
    assert np.array_equal(za, Zp.numpy())
    _close_to_oracle(za, oracle.embed(e, Y, K, weights=w, laplacian=lap))


def test_multi_label_equals_single_passes(gee, weighted_rmat):
    n, e, w, _, _ = weighted_rmat
    L, K = 3, 6
    Ys = np.stack([graphgen.labels(n, K, seed=70 + l, frac_unlabeled=0.1) for l in range(L)])
    with gee.Graph(_dev(e), n, weights=_dev(w)) as g:
        Z = g.embed_multi(_dev(Ys), K, deterministic=True).cpu().numpy()
        for l in range(L):
            one = g.embed(_dev(Ys[l]), K, deterministic=True).cpu().numpy()
            assert np.array_equal(Z[:, l * K:(l + 1) * K], one), l


def test_edge_list_call_matches_resident_graph(gee, weighted_rmat):
    n, e, w, e2, w2 = weighted_rmat
    K = 9
    Y = graphgen.labels(n, K, seed=80, frac_unlabeled=0.2)
    z_list = gee.embed(_dev(e2), _dev(Y), K, weights=_dev(w2), deterministic=True)
    with gee.Graph(_dev(e), n, weights=_dev(w)) as g:
        z_graph = g.embed(_dev(Y), K, deterministic=True)
    assert np.array_equal(z_list.cpu().numpy(), z_graph.cpu().numpy())
    z_host = gee.embed_host(e, Y, K, weights=w, deterministic=True)
    assert np.array_equal(z_host, z_graph.cpu().numpy())


def test_unit_weights_unchanged(gee, weighted_rmat):
    n, e, _, _, _ = weighted_rmat
    K = 8
    Y = graphgen.labels(n, K, seed=90)
    with gee.Graph(_dev(e), n) as g:
        z = g.embed(_dev(Y), K, deterministic=True).cpu().numpy()
    assert np.array_equal(z, oracle.embed_counts32(e, Y, K))


def test_forms_that_refuse(gee, weighted_rmat):
    n, e, w, _, _ = weighted_rmat
    K = 4
    Y = graphgen.labels(n, K, seed=91)
    for strategy in ("atomic", "private"):
        with pytest.raises(gee.GeeError) as ei:
            gee.embed(_dev(e), _dev(Y), K, weights=_dev(w), strategy=strategy,
                      deterministic=True)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
    Ys = np.stack([graphgen.labels(n, K, seed=92 + l) for l in range(8)])
    with gee.Graph(_dev(e), n, weights=_dev(w)) as g:
        with pytest.raises(gee.GeeError) as ei:
            g.embed_multi(_dev(Ys), K, deterministic=True)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
        # without weights the multi-label form is exact counts: accepted
    with gee.Graph(_dev(e), n) as g:
        g.embed_multi(_dev(Ys), K, deterministic=True)


def test_wide_rows_of_fixed_point_cells(gee, weighted_rmat):
    """4 vectors of K = 255 (1,020 columns of 8-byte cells): the kernels
    take fewer groups / warps so their accumulators fit, and the result is
    still each vector's own deterministic pass."""
    n, e, w, _, _ = weighted_rmat
    L, K = 4, 255
    Ys = np.stack([graphgen.labels(n, K, seed=95 + l, frac_unlabeled=0.1) for l in range(L)])
    with gee.Graph(_dev(e), n, weights=_dev(w)) as g:
        Z = g.embed_multi(_dev(Ys), K, deterministic=True).cpu().numpy()
        for l in (0, L - 1):
            one = g.embed(_dev(Ys[l]), K, deterministic=True).cpu().numpy()
            assert np.array_equal(Z[:, l * K:(l + 1) * K], one), l
    _close_to_oracle(Z[:, :K], oracle.embed(e, Ys[0], K, weights=w))
