"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Unit weights without the Laplacian: bit-exact against RN32(C / n_k).
Float weights and the Laplacian variant: |Z - Z64| <= 1e-5 |Z64| wherever
Z64 != 0 and Z == 0 exactly where Z64 == 0 (all weights are positive, so no
cancellation); the largest relative and absolute errors are printed.
"""
import numpy as np
import pytest

import graphgen
import oracle
from tests import _pins

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
STRATEGIES = ["atomic", "private", "segmented", "binned"]


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


def assert_weighted_close(got, want, what=""):
    got = np.asarray(got, np.float64)
    nz = want != 0
    assert np.all(got[~nz] == 0), f"{what}: nonzero where the oracle has 0"
    if nz.any():
        rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
        worst = rel.max()
        print(f"{what}: max rel err {worst:.3e}, max abs err "
              f"{np.abs(got - want).max():.3e}")
        assert worst <= REL_TOL, f"{what}: rel err {worst:.3e} > {REL_TOL}"


def run_all_paths(gee, edges, Y, K, weights=None, laplacian=False, strategies=STRATEGIES):
    """Z from every edge-list strategy and from a resident graph."""
    e_d, y_d = _dev(edges.reshape(-1, 2)), _dev(Y)
    w_d = None if weights is None else _dev(weights)
    out = {}
    for st in strategies:
        out[st] = gee.embed(e_d, y_d, K, weights=w_d, laplacian=laplacian,
                            strategy=st).cpu().numpy()
    with gee.Graph(e_d, Y.size, weights=w_d) as g:
        out["graph"] = g.embed(y_d, K, laplacian=laplacian).cpu().numpy()
    return out


def check_case(gee, edges, Y, K, weights=None, laplacian=False, what=""):
    edges = np.asarray(edges, np.int32).reshape(-1, 2)
    Y = np.asarray(Y, np.int32)
    outs = run_all_paths(gee, edges, Y, K, weights, laplacian)
    if weights is None and not laplacian:
        want = oracle.embed_counts32(edges, Y, K)
        for name, got in outs.items():
            assert got.dtype == np.float32
            mism = np.argwhere(got != want)
            assert mism.size == 0, f"{what}/{name}: {len(mism)} cells differ, first {mism[:3]}"
    else:
        want = oracle.embed(edges, Y, K, weights=weights, laplacian=laplacian)
        for name, got in outs.items():
            assert_weighted_close(got, want, f"{what}/{name}")


@pytest.mark.parametrize("case", _pins.load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(gee, case):
    w = None if case["weights"] is None else np.asarray(case["weights"], np.float32)
    check_case(gee, case["edges"], case["Y"], case["K"], w, case["laplacian"], case["name"])


def test_tiny_sbm_count_path_bit_exact(gee, tiny_sbm_graph):
    edges, Y = tiny_sbm_graph
    check_case(gee, edges, Y, 5, what="sbm")


def test_tiny_sbm_weighted_and_laplacian(gee, tiny_sbm_graph):
    edges, Y = tiny_sbm_graph
    w = graphgen.weights(edges.shape[0], seed=11)
    check_case(gee, edges, Y, 5, weights=w, what="sbm-w")
    check_case(gee, edges, Y, 5, laplacian=True, what="sbm-lap")
    check_case(gee, edges, Y, 5, weights=w, laplacian=True, what="sbm-w-lap")


RANDOM_CASES = [
    # n, s, K, frac_unlabeled
    (1, 0, 1, 0.0),
    (1, 5, 3, 0.0),          # all self-loops on one node
    (2, 1, 2, 0.5),
    (37, 1001, 5, 0.3),      # ragged: odd edge count, n*K not a multiple of 4
    (1000, 3, 50, 0.1),      # mostly isolated nodes
    (5000, 50001, 20, 0.1),  # several row tiles, ragged tail
    (3001, 40000, 255, 0.0), # K at its maximum
    (4000, 30000, 1, 0.0),   # K = 1
    (500, 20000, 7, 1.0),    # nothing labelled
    (200, 30000, 7, 0.1),    # every row above the hub threshold, one chunk
    (300, 40000, 255, 0.0),  # hub rows with K at its maximum
    (64, 200000, 3, 0.0),    # hub rows of several chunks, tiny K
]


@pytest.mark.parametrize("n,s,K,frac", RANDOM_CASES)
@pytest.mark.parametrize("weighted", [False, True])
def test_random_multigraphs(gee, n, s, K, frac, weighted):
    edges = graphgen.random_graph(n, s, seed=n * 7 + s)
    Y = graphgen.labels(n, K, seed=n + K, frac_unlabeled=frac)
    w = graphgen.weights(s, seed=s + 3) if weighted else None
    check_case(gee, edges, Y, K, weights=w, what=f"rand{n}x{s}")
    if weighted:
        check_case(gee, edges, Y, K, weights=w, laplacian=True, what=f"rand{n}x{s}-lap")


@pytest.fixture(scope="module")
def rmat16():
    """R-MAT scale 16, 2^20 edges: hub rows of many 2,048-arc chunks (the
    largest has more than 16,384 arcs)."""
    n = 1 << 16
    edges = graphgen.rmat_edges(16, n, 0, 1 << 20, seed=21)
    deg = np.bincount(edges.ravel(), minlength=n)
    assert deg.max() > 4 * 4096
    return edges, n


# K <= 63: the hub kernel's label copy holds 6-bit codes (63 = unknown);
# K = 63 is the largest such K, K = 64 the smallest with byte labels
@pytest.mark.parametrize("K,frac", [(20, 0.1), (50, 0.0), (3, 0.5), (63, 0.2), (64, 0.2)])
def test_rmat_with_hub_rows(gee, rmat16, K, frac):
    edges, n = rmat16
    Y = graphgen.labels(n, K, seed=K, frac_unlabeled=frac)
    check_case(gee, edges, Y, K, what=f"rmat16-K{K}")


def test_rmat_weighted_with_hub_rows(gee, rmat16):
    edges, n = rmat16
    K = 20
    Y = graphgen.labels(n, K, seed=99, frac_unlabeled=0.1)
    w = graphgen.weights(edges.shape[0], seed=98)
    check_case(gee, edges, Y, K, weights=w, what="rmat16-w")
    check_case(gee, edges, Y, K, weights=w, laplacian=True, what="rmat16-w-lap")


def test_unaligned_device_pointers(gee):
    """Edge and label arrays that start off a 16-byte boundary take the
    scalar paths of the streaming kernels."""
    import torch
    n, s, K = 777, 9999, 6
    edges = graphgen.random_graph(n, s, seed=5)
    Y = graphgen.labels(n, K, seed=6, frac_unlabeled=0.2)
    big_e = torch.zeros((s + 1, 2), dtype=torch.int32, device="cuda")
    big_e[1:] = _dev(edges)
    big_y = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    big_y[1:] = _dev(Y)
    e_d, y_d = big_e[1:], big_y[1:]
    assert e_d.data_ptr() % 16 != 0 and y_d.data_ptr() % 16 != 0
    want = oracle.embed_counts32(edges, Y, K)
    for st in STRATEGIES:
        got = gee.embed(e_d, y_d, K, strategy=st).cpu().numpy()
        assert np.array_equal(got, want), st
    out = torch.full((n * K + 1,), 7.0, device="cuda")[1:].view(n, K)
    got = gee.embed(e_d, y_d, K, strategy="atomic", out=out).cpu().numpy()
    assert np.array_equal(got, want)


def test_resident_graph_unaligned_output(gee, rmat16):
    """A Z that starts 4, 8 or 12 bytes past a 16-byte boundary: the row
    tiles' vector stores realign on the address, results are unchanged."""
    import torch
    edges, n = rmat16
    K = 7
    Y = graphgen.labels(n, K, seed=31, frac_unlabeled=0.1)
    want = oracle.embed_counts32(edges, Y, K)
    with gee.Graph(_dev(edges), n) as g:
        for shift in (1, 2, 3):
            buf = torch.full((n * K + 4,), 9.0, device="cuda")
            Z = buf[shift:shift + n * K].view(n, K)
            g.embed(_dev(Y), K, out=Z)
            assert np.array_equal(Z.cpu().numpy(), want), shift
            assert torch.all(buf[:shift] == 9.0) and torch.all(buf[shift + n * K:] == 9.0)
    for shift in (1, 3):
        buf = torch.full((n * K + 4,), 9.0, device="cuda")
        Z = buf[shift:shift + n * K].view(n, K)
        gee.embed(_dev(edges), _dev(Y), K, strategy="segmented", out=Z)
        assert np.array_equal(Z.cpu().numpy(), want), shift


def test_repeated_calls(gee, tiny_sbm_graph):
    """Unit weights: every call gives the same bits.  Float weights: the
    shared-memory float atomics may add in a different order from call to
    call, so repeated results agree to the stated tolerance, not bitwise."""
    import torch
    edges, Y = tiny_sbm_graph
    e_d, y_d = _dev(edges), _dev(Y)
    w_d = _dev(graphgen.weights(edges.shape[0], seed=2))
    with gee.Graph(e_d, Y.size) as g:
        assert torch.equal(g.embed(y_d, 5), g.embed(y_d, 5))
    with gee.Graph(e_d, Y.size, weights=w_d) as g:
        a = g.embed(y_d, 5).cpu().numpy()
        b = g.embed(y_d, 5).cpu().numpy()
        assert_weighted_close(a, b.astype(np.float64), "repeat-weighted")
    c = gee.embed(e_d, y_d, 5, strategy="atomic")
    d = gee.embed(e_d, y_d, 5, strategy="atomic")
    assert torch.equal(c, d)


def test_histogram(gee):
    n, K = 100003, 37
    Y = graphgen.labels(n, K, seed=8, frac_unlabeled=0.25)
    got = gee.histogram(_dev(Y), K).cpu().numpy()
    assert np.array_equal(got, oracle.class_counts(Y, K))


def test_host_entry_points(gee, tiny_sbm_graph):
    edges, Y = tiny_sbm_graph
    want = oracle.embed_counts32(edges, Y, 5)
    got = gee.embed_host(edges, Y, 5)
    assert np.array_equal(got, want)
    with gee.Graph(_dev(edges), Y.size) as g:
        assert np.array_equal(g.embed_host(Y, 5), want)
        info = g.info()
        assert info["n"] == Y.size and info["s"] == edges.shape[0]


def test_graph_host_entry_point_writes_pinned_output_directly(gee, rmat16):
    """gee_embed_graph_host with a page-locked Z (written by the pass itself)
    and a pageable Z (copied after it) gives the oracle's result; on a label
    error the page-locked Z is left untouched."""
    import torch
    edges, n = rmat16
    K = 9
    Y = graphgen.labels(n, K, seed=41, frac_unlabeled=0.1)
    want = oracle.embed_counts32(edges, Y, K)
    Zp = torch.full((n, K), 3.0).pin_memory()
    Yp = torch.from_numpy(Y).pin_memory()
    with gee.Graph(_dev(edges), n) as g:
        g.embed_host(Yp, K, out=Zp)
        assert np.array_equal(Zp.numpy(), want)
        assert np.array_equal(g.embed_host(Y, K), want)           # pageable
        bad = Y.copy()
        bad[n // 2] = K
        Zp.fill_(3.0)
        with pytest.raises(gee.GeeError) as ei:
            g.embed_host(torch.from_numpy(bad).pin_memory(), K, out=Zp)
        assert ei.value.name == "GEE_ERR_LABEL_RANGE"
        assert torch.all(Zp == 3.0)


def test_relabeling_a_resident_graph(gee, rmat16):
    """Many label vectors on one resident graph, each equal to its own
    oracle result (the unsupervised-GEE re-labeling loop)."""
    edges, n = rmat16
    with gee.Graph(_dev(edges), n) as g:
        for seed in range(3):
            K = 4 + 7 * seed
            Y = graphgen.labels(n, K, seed=1000 + seed, frac_unlabeled=0.1 * seed)
            got = g.embed(_dev(Y), K).cpu().numpy()
            assert np.array_equal(got, oracle.embed_counts32(edges, Y, K))


@pytest.mark.parametrize("L,K", [(2, 5), (3, 50), (4, 255), (7, 9),
                                 (8, 3), (16, 64), (32, 20), (33, 31),
                                 (64, 16), (256, 4)])
def test_multi_label_pass_equals_single_passes(gee, rmat16, L, K):
    """L label vectors in one pass (W widened to L*K columns): each block of
    K columns equals the oracle's embedding for that vector.  Covers both
    forms of the pass (one lane per arc below 8 vectors, one lane per label
    vector from 8 on), one and several blocks of 32 vectors, odd and even K,
    and the 1,024-column limit."""
    import torch
    edges, n = rmat16
    Ys = np.stack([graphgen.labels(n, K, seed=500 + l, frac_unlabeled=0.05 * (l % 3))
                   for l in range(L)])
    with gee.Graph(_dev(edges), n) as g:
        Z = g.embed_multi(_dev(Ys), K).cpu().numpy()
    assert Z.shape == (n, L * K)
    for l in (0, L // 2, L - 1):
        want = oracle.embed_counts32(edges, Ys[l], K)
        assert np.array_equal(Z[:, l * K:(l + 1) * K], want), l


@pytest.mark.parametrize("L,K", [(5, 7), (12, 6), (12, 8), (40, 3), (33, 4)])
def test_multi_label_weighted_laplacian(gee, L, K):
    """Weighted and Laplacian multi-label passes on an R-MAT graph whose hub
    rows span several chunks; from 8 vectors on the pass sums each cell in
    one lane, so repeated calls agree bit for bit."""
    n, s = 5000, 150000
    edges = graphgen.rmat_edges(13, n, 0, s, seed=61)
    assert np.bincount(edges.ravel(), minlength=n).max() > 2 * 2048
    w = graphgen.weights(s, seed=62)
    Ys = np.stack([graphgen.labels(n, K, seed=63 + l, frac_unlabeled=0.1) for l in range(L)])
    with gee.Graph(_dev(edges), n, weights=_dev(w)) as g:
        for lap in (False, True):
            Z = g.embed_multi(_dev(Ys), K, laplacian=lap).cpu().numpy()
            for l in sorted({0, 1, L // 2, L - 1}):
                want = oracle.embed(edges, Ys[l], K, weights=w, laplacian=lap)
                assert_weighted_close(Z[:, l * K:(l + 1) * K], want, f"multi-{l}-{lap}")
            if L >= 8:
                again = g.embed_multi(_dev(Ys), K, laplacian=lap).cpu().numpy()
                assert np.array_equal(Z.view(np.uint32), again.view(np.uint32))


def test_multi_label_unaligned_output(gee, rmat16):
    """A Z that is not 16-byte aligned takes the transposing write of the
    multi-label pass; the result is the same as with an aligned Z."""
    import torch
    edges, n = rmat16
    L, K = 16, 8
    Ys = np.stack([graphgen.labels(n, K, seed=900 + l, frac_unlabeled=0.1)
                   for l in range(L)])
    with gee.Graph(_dev(edges), n) as g:
        aligned = g.embed_multi(_dev(Ys), K).cpu().numpy()
        buf = torch.empty(n * L * K + 1, dtype=torch.float32, device="cuda")
        Z = buf[1:].view(n, L * K)
        g.embed_multi(_dev(Ys), K, out=Z)
        assert np.array_equal(Z.cpu().numpy(), aligned)
    want = oracle.embed_counts32(edges, Ys[L - 1], K)
    assert np.array_equal(aligned[:, (L - 1) * K:], want)


def test_multi_label_limits(gee, tiny_sbm_graph):
    edges, Y = tiny_sbm_graph
    with gee.Graph(_dev(edges), Y.size) as g:
        Ys = np.stack([Y] * 5)
        with pytest.raises(gee.GeeError) as ei:
            g.embed_multi(_dev(Ys), 255)  # 5 * 255 columns > 1024
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
        Ys[3, 17] = 9
        with pytest.raises(gee.GeeError) as ei:
            g.embed_multi(_dev(Ys), 5)
        assert ei.value.name == "GEE_ERR_LABEL_RANGE"


@pytest.mark.parametrize("K", [1, 3, 9, 50])
@pytest.mark.parametrize("variant", ["unit", "weighted", "laplacian"])
def test_graph_host_direct_write_hub_rows_and_offsets(gee, rmat16, K, variant):
    """The direct-write form of gee_embed_graph_host writes light rows from
    one kernel and hub rows from another at the same time: every cell of a
    page-locked Z (placed at a float offset that leaves every line
    alignment) gets its value, and no float around it changes.  Unit
    weights: the oracle bit for bit; float weights (shared-memory float
    atomics, so the summation order varies between calls): the oracle
    within 1e-5."""
    import torch
    edges, n = rmat16
    w = graphgen.weights(edges.shape[0], seed=43) if variant != "unit" else None
    lap = variant == "laplacian"
    Y = graphgen.labels(n, K, seed=44 + K, frac_unlabeled=0.2)
    for shift in (0, 5):
        buf = torch.full((n * K + 64,), float("nan"), dtype=torch.float32).pin_memory()
        Zp = buf[shift:shift + n * K].view(n, K)
        with gee.Graph(_dev(edges), n, weights=None if w is None else _dev(w)) as g:
            g.embed_host(torch.from_numpy(Y).pin_memory(), K, laplacian=lap, out=Zp)
        got = Zp.numpy()
        if w is None:
            assert np.array_equal(got, oracle.embed_counts32(edges, Y, K)), shift
        else:
            assert_weighted_close(got, oracle.embed(edges, Y, K, weights=w, laplacian=lap),
                                  f"host {variant} K={K} shift={shift}")
        rest = torch.cat([buf[:shift], buf[shift + n * K:]])
        assert torch.all(torch.isnan(rest)), shift


def test_kept_tile_splits_many_column_counts(gee, rmat16):
    """A resident graph keeps the row-tile split of the first 8 column
    counts it is embedded with and splits per call after that: twelve K in
    turn (device and page-locked host Z, which split differently), then the
    first ones again from the kept splits -- each equal to the oracle."""
    import torch
    edges, n = rmat16
    with gee.Graph(_dev(edges), n) as g:
        for rnd in range(2):
            for K in range(1, 13) if rnd == 0 else (1, 2, 3):
                Y = graphgen.labels(n, K, seed=300 + 17 * K + rnd, frac_unlabeled=0.2)
                want = oracle.embed_counts32(edges, Y, K)
                assert np.array_equal(g.embed(_dev(Y), K).cpu().numpy(), want), (rnd, K)
                Zp = torch.empty((n, K), dtype=torch.float32).pin_memory()
                g.embed_host(torch.from_numpy(Y).pin_memory(), K, out=Zp)
                assert np.array_equal(Zp.numpy(), want), (rnd, K)
