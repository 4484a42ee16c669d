"""gee_embed_batch through the C ABI: every problem of a batch equals its own
oracle result (bit for bit with unit weights, 1e-5 relative with float
weights), whatever the mix of sizes, K and weights, and a failing problem
does not disturb the others."""
import ctypes

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
    assert np.all(got[~nz] == 0), what
    if nz.any():
        rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        assert rel.max() <= REL_TOL, f"{what}: {rel.max():.3e}"


def _mixed_problems(count, seed):
    """Planted-partition graphs of mixed sizes (including empty ones), K in
    2..32 plus the extremes 1 and 255, some weighted, some with unknown
    labels."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(30000))))
        K = int(rng.integers(2, 33))
        if i % 11 == 3:
            K = 1
        if i % 13 == 5:
            K = 255
        K = min(K, n)
        deg = rng.uniform(2, 40)
        s = int(n * deg / 2)
        if i % 17 == 7:
            s = 0
        edges = graphgen.planted_edges(n, K, s, 10.0, seed=1000 + i)
        Y = graphgen.planted_labels(n, K)
        if i % 3 == 1:
            Y = graphgen.labels(n, K, seed=2000 + i, frac_unlabeled=0.2)
        w = graphgen.weights(s, seed=3000 + i) if i % 2 == 0 else None
        out.append((edges, Y, K, w))
    return out


@pytest.mark.parametrize("strategy", ["atomic", "binned"])
def test_mixed_batch_matches_oracle(gee, strategy):
    """Both edge passes of a batch: pushed atomics and binned records."""
    probs = _mixed_problems(60, seed=1)
    dev = [dict(edges=_dev(e), Y=_dev(Y), K=K, weights=None if w is None else _dev(w))
           for e, Y, K, w in probs]
    Zs = gee.embed_batch(dev, strategy=strategy)
    for i, ((e, Y, K, w), Z) in enumerate(zip(probs, Zs)):
        got = Z.cpu().numpy()
        if w is None:
            assert np.array_equal(got, oracle.embed_counts32(e, Y, K)), i
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")


@pytest.mark.parametrize("strategy", ["atomic", "binned"])
def test_batch_equals_single_calls(gee, strategy):
    """Unit weights: the batch gives the same bits as one gee_embed call per
    problem; a second run of the batch gives them again."""
    probs = [p for p in _mixed_problems(40, seed=2) if p[3] is None]
    dev = [dict(edges=_dev(e), Y=_dev(Y), K=K) for e, Y, K, _ in probs]
    Zs = [Z.cpu().numpy() for Z in gee.embed_batch(dev, strategy=strategy)]
    again = [Z.cpu().numpy() for Z in gee.embed_batch(dev, strategy=strategy)]
    for q, Z, Z2 in zip(dev, Zs, again):
        single = gee.embed(q["edges"], q["Y"], q["K"], strategy="atomic").cpu().numpy()
        assert np.array_equal(Z, single)
        assert np.array_equal(Z, Z2)


@pytest.mark.parametrize("strategy", ["atomic", "binned"])
def test_large_and_tiny_problems_in_one_batch(gee, strategy):
    """A problem spanning many chunks of every kind between tiny ones."""
    n, s, K = 150_000, 1_500_000, 13
    big = (graphgen.rmat_edges(18, n, 0, s, seed=5),
           graphgen.labels(n, K, seed=6, frac_unlabeled=0.1), K)
    tiny = [(graphgen.random_graph(7, 11, seed=i), graphgen.labels(7, 3, seed=i), 3)
            for i in range(5)]
    probs = tiny[:2] + [big] + tiny[2:]
    Zs = gee.embed_batch([dict(edges=_dev(e), Y=_dev(Y), K=K) for e, Y, K in probs],
                         strategy=strategy)
    for (e, Y, K), Z in zip(probs, Zs):
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(e, Y, K))


@pytest.mark.parametrize("strategy", ["atomic", "binned"])
def test_failing_problems_leave_the_rest_intact(gee, strategy):
    import torch
    probs = _mixed_problems(8, seed=3)
    dev = []
    for e, Y, K, w in probs:
        Yd = _dev(Y)
        dev.append(dict(edges=_dev(e), Y=Yd, K=K, weights=None if w is None else _dev(w),
                        out=torch.full((Y.size, K), 5.0, device="cuda")))
    bad_label, bad_node = 2, 5
    dev[bad_label]["Y"][0] = dev[bad_label]["K"]          # label == K
    assert probs[bad_node][0].shape[0] > 0
    dev[bad_node]["edges"][0, 1] = probs[bad_node][1].size  # endpoint == n
    Zs, codes = gee.embed_batch(dev, strategy=strategy, raise_on_error=False)
    names = [gee.STATUS_NAMES[c] for c in codes]
    assert names[bad_label] == "GEE_ERR_LABEL_RANGE"
    assert names[bad_node] == "GEE_ERR_NODE_RANGE"
    for i, ((e, Y, K, w), Z) in enumerate(zip(probs, Zs)):
        got = Z.cpu().numpy()
        if i in (bad_label, bad_node):
            assert np.all(got == 5.0), f"problem {i} was modified"
            continue
        assert names[i] == "GEE_OK"
        if w is None:
            assert np.array_equal(got, oracle.embed_counts32(e, Y, K)), i
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")
    with pytest.raises(gee.GeeError) as ei:
        gee.embed_batch(dev, strategy=strategy)
    assert ei.value.name == "GEE_ERR_LABEL_RANGE"


def test_empty_batch_and_argument_errors(gee):
    lib = gee.load()
    from paper_2402_04403_gb300 import _lib
    assert lib.gee_embed_batch(None, 0, None, None, None) == 0
    assert gee.STATUS_NAMES[lib.gee_embed_batch(None, -1, None, None, None)] == \
        "GEE_ERR_INVALID_ARG"
    arr = (_lib.Problem * 1)()
    arr[0].K = 0
    st = (ctypes.c_int * 1)()
    assert gee.STATUS_NAMES[lib.gee_embed_batch(arr, 1, st, None, None)] == \
        "GEE_ERR_INVALID_ARG"
    assert gee.STATUS_NAMES[st[0]] == "GEE_ERR_INVALID_ARG"


def test_binned_batch_over_many_tiles(gee):
    """Enough problems that the binned sequence spans many row tiles and
    coarse bins, weighted and unit problems mixed (all summed in float),
    each equal to its oracle result."""
    rng = np.random.default_rng(9)
    probs = []
    for i in range(40):
        n = int(rng.integers(20_000, 200_000))
        K = int(rng.integers(2, 60))
        s = int(n * rng.uniform(2, 10))
        e = graphgen.rmat_edges(int(np.ceil(np.log2(n))), n, 0, s, seed=700 + i)
        Y = graphgen.labels(n, K, seed=800 + i, frac_unlabeled=0.1)
        w = graphgen.weights(s, seed=900 + i) if i % 3 == 0 else None
        probs.append((e, Y, K, w))
    dev = [dict(edges=_dev(e), Y=_dev(Y), K=K, weights=None if w is None else _dev(w))
           for e, Y, K, w in probs]
    Zs = gee.embed_batch(dev, strategy="binned")
    for i, ((e, Y, K, w), Z) in enumerate(zip(probs, Zs)):
        got = Z.cpu().numpy()
        if w is None:
            assert np.array_equal(got, oracle.embed_counts32(e, Y, K)), i
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")


def test_many_tiny_problems(gee):
    """Thousands of problems of a few nodes each (many problems per chunk of
    work, so their clear, add and finish items interleave closely), each
    equal to its oracle result."""
    rng = np.random.default_rng(21)
    probs = []
    for i in range(3000):
        n = int(rng.integers(1, 60))
        K = int(rng.integers(1, min(n, 8) + 1))
        s = int(rng.integers(0, 4 * n + 1))
        e = rng.integers(0, n, size=(s, 2), dtype=np.int32)
        Y = rng.integers(-1, K, size=n, dtype=np.int32)
        w = graphgen.weights(s, seed=5000 + i) if i % 2 == 0 and s > 0 else None
        probs.append((e, Y, K, w))
    dev = [dict(edges=_dev(e), Y=_dev(Y), K=K, weights=None if w is None else _dev(w))
           for e, Y, K, w in probs]
    Zs = gee.embed_batch(dev, strategy="atomic")
    for i, ((e, Y, K, w), Z) in enumerate(zip(probs, Zs)):
        got = Z.cpu().numpy()
        if w is None:
            assert np.array_equal(got, oracle.embed_counts32(e, Y, K)), i
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")



@pytest.mark.parametrize("strategy", ["atomic", "binned"])
def test_outputs_packed_at_any_offset(gee, strategy):
    """The problems' Z are consecutive slices of one buffer, so most start
    off a 16-byte boundary (the finishing pass then has a scalar head and
    tail around its 16-byte body); each equals its oracle result and the
    guard cells between and after them are untouched."""
    import torch
    probs = _mixed_problems(12, seed=41)
    sizes = [Y.size * K for _, Y, K, _ in probs]
    offs = np.concatenate([[1], np.cumsum(np.asarray(sizes) + 1) + 1])
    buf = torch.full((int(offs[-1]) + 3,), 7.0, device="cuda")
    dev = []
    for (e, Y, K, w), o in zip(probs, offs):
        out = buf[int(o):int(o) + Y.size * K].view(Y.size, K)
        dev.append(dict(edges=_dev(e), Y=_dev(Y), K=K,
                        weights=None if w is None else _dev(w), out=out))
    gee.embed_batch(dev, strategy=strategy)
    host = buf.cpu().numpy()
    mask = np.ones(host.size, bool)
    for i, ((e, Y, K, w), o) in enumerate(zip(probs, offs)):
        got = host[int(o):int(o) + Y.size * K].reshape(Y.size, K)
        mask[int(o):int(o) + Y.size * K] = False
        if w is None and strategy == "atomic":
            assert np.array_equal(got, oracle.embed_counts32(e, Y, K)), i
        else:
            _close(got, oracle.embed(e, Y, K, weights=w), f"problem {i}")
    assert np.all(host[mask] == 7.0), "a guard cell was written"
