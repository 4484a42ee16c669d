"""Parity at the full sizes the benchmark times, on sampled rows.

The paper-scale R-MAT graph (n = 65.6 M nodes, s = 1.8 B unit-weight edges,
K = 50; all labelled, then 90 % unlabelled) goes through the three calls the
benchmark times: the resident-graph pass with device Y and Z, the same pass
writing a page-locked host Z, and the one-shot edge-list call.  R-MAT scale
24 with float weights in (0, 1] (K = 20, 10 % unlabelled) goes through the
resident pass plain, in Laplacian form and deterministic, through the
widened pass with 32 label vectors, and through the one-shot edge-list call
with each scatter strategy (plain and Laplacian).  A weighted batch holds a
hub-heavy R-MAT graph (scale 22) beside small planted-partition graphs.  An
R-MAT graph of 2^25 nodes checks the hub kernel's 6-bit label codes at
K = 63 against its byte labels at K = 64.

Rows checked: the 64 of highest degree (hub rows of many chunks) and 4,096
random ones; the oracle computes just those rows in one pass over the edge
list.  Unit weights: bit-exact against RN32(C / n_k) of the exact counts.
Float weights: |Z - Z64| <= 1e-5 |Z64|, and zero exactly where Z64 is zero.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

REL_TOL = 1e-5
RANDOM_ROWS = 4096


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


def _sample_rows(ed, n, seed):
    """The 64 highest-degree nodes and RANDOM_ROWS random ones.  Degrees
    are counted with torch on the device, in slices of the edge list; they
    only choose which rows to check."""
    import torch
    deg = torch.zeros(n, dtype=torch.int64, device=ed.device)
    step = 1 << 26
    for i in range(0, ed.shape[0], step):
        deg += torch.bincount(ed[i:i + step].reshape(-1).long(), minlength=n)
    top = torch.topk(deg, 64).indices.cpu().numpy()
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([top, rng.integers(0, n, RANDOM_ROWS)]))


def _oracle_rows_parallel(calls):
    """Run oracle.embed_rows calls side by side in threads (the C oracle
    runs without the interpreter lock); results in call order."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(calls)) as ex:
        futs = [ex.submit(oracle.embed_rows, *a, **kw) for a, kw in calls]
        return [f.result() for f in futs]


def _rows_of(Z, r):
    """Rows r of a device or host Z as a float32 numpy array."""
    import torch
    if Z.is_cuda:
        return Z[torch.from_numpy(r).to(Z.device)].cpu().numpy()
    return Z.numpy()[r]


def _assert_close(got, z64, what):
    """Within REL_TOL of the FP64 oracle where it is non-zero, exactly zero
    where it is zero; prints the max relative and absolute errors."""
    nz = z64 != 0
    assert np.all(got[~nz] == 0), what
    err = np.abs(got[nz].astype(np.float64) - z64[nz])
    rel = err / np.abs(z64[nz])
    print(f"{what}: max rel err {rel.max():.3e}, max abs err {err.max():.3e}")
    assert rel.max() <= REL_TOL, f"{what}: rel err {rel.max():.3e}"


def test_paper_scale_unit_weights(gee):
    import torch
    n, s, K, scale, seed = 65_600_000, 1_800_000_000, 50, 26, 3
    dev = torch.device("cuda", 0)
    ed = graphgen.rmat_edges_device(scale, n, 0, s, seed, device=dev)
    rows = _sample_rows(ed, n, seed=17)
    e_h = ed.cpu().numpy()
    label_sets = [graphgen.labels_device(n, K, seed + 1, frac, device=dev)
                  for frac in (0.0, 0.9)]
    Y_hs = [Yd.cpu().numpy() for Yd in label_sets]
    got = _oracle_rows_parallel([((e_h, Y_h, K, rows), dict(with_counts=True))
                                 for Y_h in Y_hs])
    wants = [(r, oracle.round_counts(C, oracle.class_counts(Y_h, K)))
             for (r, _, C), Y_h in zip(got, Y_hs)]
    del e_h, got
    Z = torch.empty((n, K), dtype=torch.float32, device=dev)
    Zh = torch.empty((n, K), dtype=torch.float32).pin_memory()
    with gee.Graph(ed, n) as g:
        for Yd, (r, want) in zip(label_sets, wants):
            g.embed(Yd, K, out=Z)
            assert np.array_equal(_rows_of(Z, r), want), "resident pass"
            g.embed_host(Yd.cpu().pin_memory(), K, out=Zh)
            assert np.array_equal(_rows_of(Zh, r), want), "resident pass, host Z"
    for Yd, (r, want) in zip(label_sets, wants):
        gee.embed(ed, Yd, K, out=Z)
        assert np.array_equal(_rows_of(Z, r), want), "one-shot call"


def test_hub_label_codes_at_their_limits(gee):
    """From 2^25 nodes the hub kernel keeps its shared label copy as 6-bit
    codes (63 = unknown) when K <= 63: K = 63, the largest such K, with a
    third of the labels unknown, and K = 64 (byte copy) on the same graph,
    each bit-exact on the sampled rows."""
    import torch
    n, s, scale, seed = 1 << 25, 1 << 27, 25, 8
    dev = torch.device("cuda", 0)
    ed = graphgen.rmat_edges_device(scale, n, 0, s, seed, device=dev)
    rows = _sample_rows(ed, n, seed=19)
    e_h = ed.cpu().numpy()
    Ks = (63, 64)
    label_sets = [graphgen.labels_device(n, K, seed + K, 1.0 / 3.0, device=dev)
                  for K in Ks]
    Y_hs = [Yd.cpu().numpy() for Yd in label_sets]
    got = _oracle_rows_parallel([((e_h, Y_h, K, rows), dict(with_counts=True))
                                 for Y_h, K in zip(Y_hs, Ks)])
    del e_h
    with gee.Graph(ed, n) as g:
        for Yd, Y_h, K, (r, _, C) in zip(label_sets, Y_hs, Ks, got):
            want = oracle.round_counts(C, oracle.class_counts(Y_h, K))
            Z = g.embed(Yd, K)
            assert np.array_equal(_rows_of(Z, r), want), f"K = {K}"
            ga = g.gathers(K)
            print(f"K = {K}: {ga['hub_shared']} hub arcs from the shared copy, "
                  f"{ga['hub_other']} gathered")
            del Z
        assert g.gathers(63)["hub_shared"] > g.gathers(64)["hub_shared"]


def test_rmat24_float_weights(gee):
    import torch
    n, s, K, scale, seed = 1 << 24, 268_435_456, 20, 24, 2
    dev = torch.device("cuda", 0)
    ed = graphgen.rmat_edges_device(scale, n, 0, s, seed, device=dev)
    wd = graphgen.weights_device(s, seed + 2, device=dev)
    Yd = graphgen.labels_device(n, K, seed + 1, 0.1, device=dev)
    rows = _sample_rows(ed, n, seed=19)
    e_h, w_h, Y_h = ed.cpu().numpy(), wd.cpu().numpy(), Yd.cpu().numpy()
    L = 32
    Ys = np.stack([graphgen.labels(n, K, seed=900 + l, frac_unlabeled=0.1) for l in range(L)])
    (r, z64), (_, z64l), (_, z64m0), (_, z64m1) = _oracle_rows_parallel(
        [((e_h, Y_h, K, rows), dict(weights=w_h)),
         ((e_h, Y_h, K, rows), dict(weights=w_h, laplacian=True)),
         ((e_h, Ys[0], K, rows), dict(weights=w_h)),
         ((e_h, Ys[L - 1], K, rows), dict(weights=w_h))])
    with gee.Graph(ed, n, weights=wd) as g:
        for lap, want in ((False, z64), (True, z64l)):
            _assert_close(_rows_of(g.embed(Yd, K, laplacian=lap), r), want,
                          f"laplacian={lap}")
            zd = g.embed(Yd, K, laplacian=lap, deterministic=True)
            _assert_close(_rows_of(zd, r), want, f"deterministic, laplacian={lap}")
        Zm = _rows_of(g.embed_multi(torch.from_numpy(Ys).to(dev), K), r)
        _assert_close(Zm[:, :K], z64m0, f"vector 0 of {L}")
        _assert_close(Zm[:, (L - 1) * K:], z64m1, f"vector {L - 1} of {L}")
    # the one-shot edge-list call, every strategy that takes this size
    # (GEE_AUTO's choice included), plain and Laplacian
    Z = torch.empty((n, K), dtype=torch.float32, device=dev)
    for strategy in ONE_SHOT_STRATEGIES:
        for lap, want in ((False, z64), (True, z64l)):
            gee.embed(ed, Yd, K, weights=wd, laplacian=lap, strategy=strategy, out=Z)
            _assert_close(_rows_of(Z, r), want, f"one-shot {strategy}, laplacian={lap}")


ONE_SHOT_STRATEGIES = ("auto", "atomic", "segmented", "binned")


def test_weighted_batch_with_a_hub_heavy_graph(gee):
    """One batch: an R-MAT scale-22 graph with float weights (n = 4.2 M,
    s = 64 M; hub rows of ~10^5 arcs, so hub cells sum ~10^4 weights each)
    and 200 small weighted planted-partition graphs.  The R-MAT problem is
    checked on its top-64 and 4,096 random rows, the small ones in full."""
    import torch
    dev = torch.device("cuda", 0)
    n, s, K, scale, seed = 1 << 22, 1 << 26, 20, 22, 5
    ed = graphgen.rmat_edges_device(scale, n, 0, s, seed, device=dev)
    wd = graphgen.weights_device(s, seed + 2, device=dev)
    Yd = graphgen.labels_device(n, K, seed + 1, 0.1, device=dev)
    rows = _sample_rows(ed, n, seed=23)
    probs = [dict(edges=ed, Y=Yd, K=K, weights=wd)]
    small = []
    rng = np.random.default_rng(seed)
    for i in range(200):
        ni = int(np.exp(rng.uniform(np.log(100), np.log(100000))))
        Ki = int(rng.integers(2, 33))
        si = int(ni * rng.uniform(5, 25))
        e = graphgen.planted_edges(ni, Ki, si, 10.0, seed=4000 + i)
        Y = graphgen.planted_labels(ni, Ki)
        w = graphgen.weights(si, seed=5000 + i)
        small.append((e, Y, Ki, w))
        probs.append(dict(edges=torch.from_numpy(e).to(dev), Y=torch.from_numpy(Y).to(dev),
                          K=Ki, weights=torch.from_numpy(w).to(dev)))
    r, z64 = oracle.embed_rows(ed.cpu().numpy(), Yd.cpu().numpy(), K, rows,
                               weights=wd.cpu().numpy())
    Zs = gee.embed_batch(probs)
    _assert_close(_rows_of(Zs[0], r), z64, "batch: R-MAT scale 22")
    worst = 0.0
    for (e, Y, Ki, w), Z in zip(small, Zs[1:]):
        want = oracle.embed(e, Y, Ki, weights=w)
        got = Z.cpu().numpy().astype(np.float64)
        nz = want != 0
        assert np.all(got[~nz] == 0)
        worst = max(worst, float((np.abs(got[nz] - want[nz]) / want[nz]).max()))
    print(f"batch: 200 small graphs, max rel err {worst:.3e}")
    assert worst <= REL_TOL
