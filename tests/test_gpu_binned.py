"""GEE_BINNED through the C ABI on graphs large enough for many row tiles
and coarse bins, against the FP64 oracle.

A row tile holds 51,200 count cells (25,600 with weights), so n * K of a
few million already spreads the records over hundreds of tiles in tens of
coarse bins; these cases still finish in the oracle within seconds.  Unit
weights: bit-exact against RN32(C / n_k).  Weights and the Laplacian:
within 1e-5 relative, exactly zero where the oracle is zero.
"""
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
    nz = want != 0
    assert np.all(got[~nz] == 0), f"{what}: nonzero where the oracle has 0"
    err = np.abs(got[nz] - want[nz])
    rel = err / np.abs(want[nz])
    print(f"{what}: max rel err {rel.max():.3e}, max abs err {err.max():.3e}")
    assert rel.max() <= REL_TOL, f"{what}: {rel.max():.3e}"


@pytest.fixture(scope="module")
def rmat20():
    """R-MAT scale 20 (ids permuted), n = 10^6, 8 M edges, float weights."""
    n, s = 1_000_000, 8_000_000
    edges = graphgen.rmat_edges(20, n, 0, s, seed=61)
    w = graphgen.weights(s, seed=62)
    return edges, w, n


@pytest.mark.parametrize("K,frac", [(20, 0.1), (50, 0.0), (255, 0.3), (1, 0.0), (3, 0.9)])
def test_many_tiles_unit_weights(gee, rmat20, K, frac):
    edges, _, n = rmat20
    Y = graphgen.labels(n, K, seed=63 + K, frac_unlabeled=frac)
    got = gee.embed(_dev(edges), _dev(Y), K, strategy="binned").cpu().numpy()
    want = oracle.embed_counts32(edges, Y, K)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} cells differ, first {bad[:3]}"


@pytest.mark.parametrize("K", [7, 50])
@pytest.mark.parametrize("laplacian", [False, True])
def test_many_tiles_weighted(gee, rmat20, K, laplacian):
    edges, w, n = rmat20
    Y = graphgen.labels(n, K, seed=70 + K, frac_unlabeled=0.1)
    got = gee.embed(_dev(edges), _dev(Y), K, weights=_dev(w), laplacian=laplacian,
                    strategy="binned").cpu().numpy()
    _close(got, oracle.embed(edges, Y, K, weights=w, laplacian=laplacian),
           f"binned K={K} laplacian={laplacian}")


def test_unit_laplacian(gee, rmat20):
    edges, _, n = rmat20
    Y = graphgen.labels(n, 12, seed=80, frac_unlabeled=0.2)
    got = gee.embed(_dev(edges), _dev(Y), 12, laplacian=True, strategy="binned").cpu().numpy()
    _close(got, oracle.embed(edges, Y, 12, laplacian=True), "binned unit Laplacian")


def test_hub_tiles(gee):
    """Two stars (hub rows of 3 M and 1 M arcs) among random edges: the hub
    tiles hold far more records than cells, which takes the warp-merged
    count path; K = 1 puts every hub record in one cell."""
    n = 400_000
    rng = np.random.default_rng(5)
    leaves_a = rng.integers(0, n, 3_000_000).astype(np.int32)
    leaves_b = rng.integers(0, n, 1_000_000).astype(np.int32)
    rand = graphgen.random_graph(n, 2_000_000, seed=6)
    edges = np.concatenate([np.stack([np.full_like(leaves_a, 17), leaves_a], 1),
                            np.stack([leaves_b, np.full_like(leaves_b, 250_000)], 1),
                            rand]).astype(np.int32)
    edges = edges[rng.permutation(edges.shape[0])]
    w = graphgen.weights(edges.shape[0], seed=7)
    for K in (1, 3, 40):
        Y = graphgen.labels(n, K, seed=8 + K, frac_unlabeled=0.05)
        got = gee.embed(_dev(edges), _dev(Y), K, strategy="binned").cpu().numpy()
        assert np.array_equal(got, oracle.embed_counts32(edges, Y, K)), K
        got = gee.embed(_dev(edges), _dev(Y), K, weights=_dev(w), strategy="binned").cpu().numpy()
        _close(got, oracle.embed(edges, Y, K, weights=w), f"hub tiles weighted K={K}")


def test_unaligned_output_and_no_edges(gee, rmat20):
    """Z starting 4 bytes past a 16-byte boundary (every tile then starts
    its rows at another offset); an empty edge list writes zeros."""
    import torch
    edges, _, n = rmat20
    K = 9
    Y = graphgen.labels(n, K, seed=90, frac_unlabeled=0.1)
    buf = torch.full((n * K + 8,), 7.0, device="cuda")
    for shift in (1, 2, 3):
        buf.fill_(7.0)
        Z = buf[shift:shift + n * K].view(n, K)
        gee.embed(_dev(edges), _dev(Y), K, strategy="binned", out=Z)
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, Y, K)), shift
        assert torch.all(buf[:shift] == 7.0) and torch.all(buf[shift + n * K:] == 7.0)
    empty = np.zeros((0, 2), np.int32)
    Z = gee.embed(_dev(empty), _dev(Y), K, strategy="binned").cpu().numpy()
    assert np.all(Z == 0)


def test_repeated_calls_and_auto_choice(gee, rmat20):
    """Back-to-back calls reuse pool scratch: the same bits each time; AUTO
    takes BINNED once Z has more than 2^24 cells."""
    edges, _, n = rmat20
    K = 20
    Y = graphgen.labels(n, K, seed=91, frac_unlabeled=0.1)
    first = gee.embed(_dev(edges), _dev(Y), K, strategy="binned").cpu().numpy()
    for _ in range(3):
        again = gee.embed(_dev(edges), _dev(Y), K, strategy="binned").cpu().numpy()
        assert np.array_equal(first, again)
    assert gee.pick_strategy(edges.shape[0], n, K) == "binned"
    assert gee.pick_strategy(edges.shape[0], n, 16) != "binned"
    assert np.array_equal(gee.embed(_dev(edges), _dev(Y), K).cpu().numpy(), first)


def test_errors_leave_z(gee, rmat20):
    """A bad label or endpoint fails the call before any Z row is written,
    with or without the separate validation pass."""
    import torch
    edges, _, n = rmat20
    K = 20
    Y = graphgen.labels(n, K, seed=92)
    Z = torch.full((n, K), 4.5, device="cuda")
    bad = Y.copy()
    bad[n - 1] = K
    with pytest.raises(gee.GeeError) as ei:
        gee.embed(_dev(edges), _dev(bad), K, strategy="binned", out=Z)
    assert ei.value.name == "GEE_ERR_LABEL_RANGE" and torch.all(Z == 4.5)
    e2 = edges.copy()
    e2[123_456, 0] = n
    for validate in (True, False):
        with pytest.raises(gee.GeeError) as ei:
            gee.embed(_dev(e2), _dev(Y), K, strategy="binned", validate_edges=validate, out=Z)
        assert ei.value.name == "GEE_ERR_NODE_RANGE" and torch.all(Z == 4.5)


def test_more_than_65536_tiles(gee):
    """K = 255 on 9 M nodes: 128 rows per tile, about 70,000 tiles, past
    the 16 bits that otherwise carry the whole tile number in a record
    (the wide record form).  Sampled rows (the 64 of highest degree and
    4,096 random ones) bit-exact against the oracle's counts."""
    import torch
    n, s, K = 9_000_000, 20_000_000, 255
    edges = graphgen.rmat_edges(24, n, 0, s, seed=95)
    Y = graphgen.labels(n, K, seed=96, frac_unlabeled=0.1)
    e_d = _dev(edges)
    Z = gee.embed(e_d, _dev(Y), K, strategy="binned")
    deg = torch.bincount(e_d.reshape(-1).long(), minlength=n)
    top = torch.topk(deg, 64).indices.cpu().numpy()
    rows = np.unique(np.concatenate(
        [top, np.random.default_rng(97).integers(0, n, 4096)]))
    r, _, C = oracle.embed_rows(edges, Y, K, rows, with_counts=True)
    want = oracle.round_counts(C, oracle.class_counts(Y, K))
    got = Z[torch.from_numpy(r).cuda()].cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,K", [(100, 5), (3000, 50), (5000, 50), (7 * 1024 - 1, 50)])
def test_tile_pairs_at_odd_counts(gee, n, K):
    """Tile records are laid out by pair of row tiles (the even tile from the
    region's start, the odd one from its end): one tile (a pair with no odd
    tile), three, five and seven tiles (the last pair half empty), unit and
    float weights and the Laplacian form, each equal to the oracle."""
    rng = np.random.default_rng(n)
    s = 20 * n
    edges = rng.integers(0, n, size=(s, 2), dtype=np.int32)
    Y = graphgen.labels(n, K, seed=n + 1, frac_unlabeled=0.1)
    w = graphgen.weights(s, seed=n + 2)
    got = gee.embed(_dev(edges), _dev(Y), K, strategy="binned").cpu().numpy()
    assert np.array_equal(got, oracle.embed_counts32(edges, Y, K))
    got = gee.embed(_dev(edges), _dev(Y), K, weights=_dev(w),
                    strategy="binned").cpu().numpy()
    _close(got, oracle.embed(edges, Y, K, weights=w), f"pairs n={n} weighted")
    got = gee.embed(_dev(edges), _dev(Y), K, weights=_dev(w), laplacian=True,
                    strategy="binned").cpu().numpy()
    _close(got, oracle.embed(edges, Y, K, weights=w, laplacian=True),
           f"pairs n={n} Laplacian")


def test_tile_pairs_across_problems(gee):
    """A binned batch numbers the row tiles of all its problems in one
    sequence, so a pair of tiles can belong to two problems: problems of
    three tiles each (and one of a single tile), unit and float weights,
    each equal to its oracle result."""
    rng = np.random.default_rng(77)
    probs = []
    for i, n in enumerate([3 * 1024 - 5, 1000, 3 * 1024, 2 * 1024 + 1, 3 * 1024 - 1]):
        K = 50
        s = 15 * n
        e = rng.integers(0, n, size=(s, 2), dtype=np.int32)
        Y = graphgen.labels(n, K, seed=300 + i, frac_unlabeled=0.2)
        w = graphgen.weights(s, seed=400 + i) if i % 2 else None
        probs.append((e, Y, K, w))
    dev = [dict(edges=_dev(e), Y=_dev(Y), K=K, weights=None if w is None else _dev(w))
           for e, Y, K, w in probs]
    Zs = gee.embed_batch(dev, strategy="binned")
    for i, ((e, Y, K, w), Z) in enumerate(zip(probs, Zs)):
        got = Z.cpu().numpy()
        if w is None:
            # a batch with any weighted problem sums every problem in float
            _close(got, oracle.embed(e, Y, K), f"problem {i}")
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")
