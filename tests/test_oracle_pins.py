"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: every expected value comes from
a hand derivation (tests/golden), a different formulation (dense product,
pairwise exact rationals, scipy's normalised Laplacian), an invariant or a
statistical expectation.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import graphgen
import oracle
from tests import _pins


def _case_arrays(case):
    edges = np.asarray(case["edges"], dtype=np.int32).reshape(-1, 2)
    w = None if case["weights"] is None else np.asarray(case["weights"], np.float32)
    return edges, w, np.asarray(case["Y"], dtype=np.int32)


@pytest.mark.parametrize("case", _pins.load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(case):
    edges, w, Y = _case_arrays(case)
    Z = oracle.embed(edges, Y, case["K"], weights=w, laplacian=case["laplacian"])
    expect = np.array([[_pins.parse_exact(x) for x in row] for row in case["Z"]])
    assert Z.shape == expect.shape
    np.testing.assert_allclose(Z, expect, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize(
    "case", [c for c in _pins.load_hand_cases()
             if c["weights"] is None and not c["laplacian"]],
    ids=lambda c: c["name"])
def test_hand_cases_exact_counts(case):
    edges, _, Y = _case_arrays(case)
    C = oracle.counts(edges, Y, case["K"])
    nk = [int((Y == k).sum()) for k in range(case["K"])]
    for u, row in enumerate(case["Z"]):
        for k, text in enumerate(row):
            got = Fraction(int(C[u, k]), nk[k]) if nk[k] else Fraction(int(C[u, k]))
            assert got == _pins.parse_fraction(text), (u, k)


def _random_case(seed, n, s, K, frac_unlabeled, weighted):
    edges = graphgen.random_graph(n, s, seed)
    Y = graphgen.labels(n, K, seed + 1, frac_unlabeled)
    w = graphgen.weights(s, seed + 2) if weighted else None
    return edges, Y, w


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("weighted", [False, True])
def test_dense_closed_form(seed, weighted):
    n, s, K = 37 + 5 * seed, 150 + 40 * seed, 1 + seed % 5
    edges, Y, w = _random_case(100 + seed, n, s, K, 0.2, weighted)
    Z = oracle.embed(edges, Y, K, weights=w)
    Zd = _pins.dense_embedding(edges, Y, K, weights=w)
    np.testing.assert_allclose(Z, Zd, rtol=1e-12, atol=1e-13)


def test_exhaustive_three_node_graphs():
    """Every edge set on 3 nodes (self-loops included) under every labelling
    with classes {-1, 0, 1}, both edge orientations: exact rationals."""
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    rng = np.random.default_rng(0)
    for mask in range(1 << len(pairs)):
        chosen = [p for b, p in enumerate(pairs) if mask >> b & 1]
        for Yt in itertools.product([-1, 0, 1], repeat=3):
            # orient each edge randomly: the result must not depend on it
            edges = [(v, u) if rng.random() < 0.5 else (u, v) for u, v in chosen]
            e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
            Y = np.asarray(Yt, dtype=np.int32)
            C = oracle.counts(e, Y, 2)
            Z = oracle.embed(e, Y, 2)
            exact = _pins.pairwise_exact(edges, list(Yt), 2)
            nk = [Yt.count(0), Yt.count(1)]
            for u in range(3):
                for k in range(2):
                    q = exact[u][k]
                    assert Fraction(int(C[u, k]), nk[k] or 1) == q
                    assert abs(Z[u, k] - float(q)) <= 1e-15 * max(1.0, float(q))


def test_exhaustive_four_node_graphs():
    """Every edge set on 4 nodes (10 pairs, self-loops included) under
    every labelling with classes {-1, 0, 1}, random orientations: counts and
    FP64 values against exact rationals computed pair by pair."""
    pairs = [(u, v) for u in range(4) for v in range(u, 4)]
    labellings = list(itertools.product([-1, 0, 1], repeat=4))
    rng = np.random.default_rng(1)
    for mask in range(1 << len(pairs)):
        chosen = [p for b, p in enumerate(pairs) if mask >> b & 1]
        edges = [(v, u) if rng.random() < 0.5 else (u, v) for u, v in chosen]
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        for Yt in labellings:
            Y = np.asarray(Yt, dtype=np.int32)
            C = oracle.counts(e, Y, 2)
            Z = oracle.embed(e, Y, 2)
            exact = _pins.pairwise_exact(edges, list(Yt), 2)
            nk = [Yt.count(0), Yt.count(1)]
            for u in range(4):
                for k in range(2):
                    q = exact[u][k]
                    assert Fraction(int(C[u, k]), nk[k] or 1) == q, (mask, Yt, u, k)
                    assert abs(Z[u, k] - float(q)) <= 1e-15 * max(1.0, float(q))


def test_exhaustive_five_node_edge_sets():
    """Every edge set on 5 nodes (15 pairs, self-loops included; 32,768
    graphs), random orientations, each under two labellings drawn from
    {-1, 0, 1}^5: exact counts and FP64 values against exact rationals
    computed pair by pair."""
    pairs = [(u, v) for u in range(5) for v in range(u, 5)]
    labellings = list(itertools.product([-1, 0, 1], repeat=5))
    rng = np.random.default_rng(6)
    for mask in range(1 << len(pairs)):
        chosen = [p for b, p in enumerate(pairs) if mask >> b & 1]
        edges = [(v, u) if rng.random() < 0.5 else (u, v) for u, v in chosen]
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        for li in rng.integers(0, len(labellings), size=2):
            Yt = labellings[li]
            Y = np.asarray(Yt, dtype=np.int32)
            C = oracle.counts(e, Y, 2)
            Z = oracle.embed(e, Y, 2)
            exact = _pins.pairwise_exact(edges, list(Yt), 2)
            nk = [Yt.count(0) or 1, Yt.count(1) or 1]
            for u in range(5):
                for k in range(2):
                    q = exact[u][k]
                    assert Fraction(int(C[u, k]), nk[k]) == q, (mask, Yt, u, k)
                    assert abs(Z[u, k] - float(q)) <= 1e-15 * max(1.0, float(q))


def _four_node_edge_sets(seed):
    """Every edge set on 4 nodes (10 pairs, self-loops included), each edge
    in a random orientation."""
    pairs = [(u, v) for u in range(4) for v in range(u, 4)]
    rng = np.random.default_rng(seed)
    for mask in range(1 << len(pairs)):
        chosen = [p for b, p in enumerate(pairs) if mask >> b & 1]
        yield mask, [(v, u) if rng.random() < 0.5 else (u, v) for u, v in chosen]


def test_exhaustive_four_node_graphs_signed_dyadic_weights():
    """Every edge set on 4 nodes with signed weights in steps of 1/8 (a
    repeated pair sums its weights; cancellation to zero happens), under
    sampled labellings with classes {-1, 0, 1, 2}: FP64 values against exact
    rationals computed pair by pair."""
    rng = np.random.default_rng(2)
    labellings = list(itertools.product([-1, 0, 1, 2], repeat=4))
    for mask, edges in _four_node_edge_sets(3):
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        w = (rng.integers(-16, 17, size=len(edges)) / 8.0).astype(np.float32)
        if len(edges) > 1 and rng.random() < 0.25:
            # a listed duplicate whose weight cancels its twin
            e = np.vstack([e, e[:1, ::-1]])
            w = np.concatenate([w, -w[:1]])
        for li in rng.choice(len(labellings), size=4, replace=False):
            Yt = labellings[li]
            Y = np.asarray(Yt, dtype=np.int32)
            Z = oracle.embed(e, Y, 3, weights=w)
            exact = _pins.pairwise_exact_weighted(e.tolist(), w, list(Yt), 3)
            for u in range(4):
                for k in range(3):
                    q = exact[u][k]
                    assert abs(Z[u, k] - float(q)) <= 1e-14 * max(1.0, abs(float(q))), \
                        (mask, Yt, u, k, Z[u, k], q)


def test_exhaustive_four_node_graphs_laplacian():
    """Every edge set on 4 nodes with non-negative weights in steps of 1/8
    (zero weights included, so some listed edges leave a degree at zero),
    Laplacian form, under sampled labellings: FP64 values against a 40-digit
    decimal evaluation of D^-1/2 A D^-1/2 W pair by pair."""
    rng = np.random.default_rng(4)
    labellings = list(itertools.product([-1, 0, 1], repeat=4))
    for mask, edges in _four_node_edge_sets(5):
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        w = (rng.integers(0, 17, size=len(edges)) / 8.0).astype(np.float32)
        for li in rng.choice(len(labellings), size=3, replace=False):
            Yt = labellings[li]
            Y = np.asarray(Yt, dtype=np.int32)
            Z = oracle.embed(e, Y, 2, weights=w, laplacian=True)
            ref = _pins.pairwise_laplacian_decimal(e.tolist(), w, list(Yt), 2)
            for u in range(4):
                for k in range(2):
                    q = float(ref[u][k])
                    assert abs(Z[u, k] - q) <= 1e-14 * max(1.0, abs(q)), \
                        (mask, Yt, u, k, Z[u, k], q)


@pytest.mark.parametrize("seed", range(4))
def test_row_and_column_sum_invariants(seed):
    n, s, K = 300, 2000, 6
    edges, Y, w = _random_case(200 + seed, n, s, K, 0.15, True)
    Z = oracle.embed(edges, Y, K, weights=w)
    nk = np.bincount(Y[Y >= 0], minlength=K).astype(np.float64)
    u, v = edges[:, 0].astype(np.int64), edges[:, 1].astype(np.int64)
    w64 = w.astype(np.float64)
    # R1: sum_k n_k Z[u,k] = weight of u's edges whose other end is labelled
    lab_v = (Y[v] >= 0).astype(np.float64)
    lab_u = (Y[u] >= 0).astype(np.float64)
    r1 = np.bincount(u, w64 * lab_v, n) + np.bincount(v, w64 * lab_u, n)
    np.testing.assert_allclose(Z @ nk, r1, rtol=1e-12, atol=1e-12)
    # R2: sum_u n_k Z[u,k] = total weighted degree of the nodes of class k
    d = np.bincount(u, w64, n) + np.bincount(v, w64, n)
    r2 = np.array([d[Y == k].sum() for k in range(K)])
    np.testing.assert_allclose(Z.sum(axis=0) * nk, r2, rtol=1e-12, atol=1e-12)


def test_single_class_is_degree_over_n():
    n, s = 500, 4000
    edges, _, w = _random_case(7, n, s, 1, 0.0, True)
    Y = np.zeros(n, np.int32)
    Z = oracle.embed(edges, Y, 1, weights=w)
    u, v = edges[:, 0].astype(np.int64), edges[:, 1].astype(np.int64)
    d = np.bincount(u, w.astype(np.float64), n) + np.bincount(v, w.astype(np.float64), n)
    np.testing.assert_allclose(Z[:, 0], d / n, rtol=1e-12, atol=1e-15)


def test_equivariance():
    n, s, K = 200, 1500, 5
    edges, Y, w = _random_case(11, n, s, K, 0.1, True)
    Z = oracle.embed(edges, Y, K, weights=w)
    C = oracle.counts(edges, Y, K)
    rng = np.random.default_rng(3)
    # edge order and orientation
    order = rng.permutation(s)
    flip = rng.random(s) < 0.5
    e2 = edges[order].copy()
    e2[flip] = e2[flip][:, ::-1]
    np.testing.assert_allclose(oracle.embed(e2, Y, K, weights=w[order]), Z,
                               rtol=1e-12, atol=1e-15)
    assert np.array_equal(oracle.counts(e2, Y, K), C)
    # class ids permuted -> columns permuted
    cp = rng.permutation(K)
    Y2 = np.where(Y >= 0, cp[np.maximum(Y, 0)], -1).astype(np.int32)
    Zc = oracle.embed(edges, Y2, K, weights=w)
    np.testing.assert_allclose(Zc[:, cp], Z, rtol=1e-12, atol=1e-15)
    # node ids permuted -> rows permuted
    p = rng.permutation(n).astype(np.int32)
    e3 = p[edges]
    Y3 = np.empty_like(Y)
    Y3[p] = Y
    Zn = oracle.embed(e3, Y3, K, weights=w)
    np.testing.assert_allclose(Zn[p], Z, rtol=1e-12, atol=1e-15)
    assert np.array_equal(oracle.counts(e3, Y3, K)[p], C)


def test_sbm_block_means(tiny_sbm_graph):
    """Tiny SBM: Z[u,k] = (neighbours of u in block k) / 2000, so block means
    are p_in (2000-1)/2000 on the diagonal and p_out off it."""
    edges, Y = tiny_sbm_graph
    K, m = 5, 2000
    n_pairs = 5 * m * (m - 1) // 2 + 10 * m * m
    mean_s = 5 * m * (m - 1) / 2 * 0.02 + 10 * m * m * 0.002
    var_s = 5 * m * (m - 1) / 2 * 0.02 * 0.98 + 10 * m * m * 0.002 * 0.998
    assert abs(edges.shape[0] - mean_s) < 5 * np.sqrt(var_s), n_pairs
    Z = oracle.embed(edges, Y, K)
    for b in range(K):
        rows = Z[Y == b]
        for k in range(K):
            if k == b:
                p, cnt = 0.02, m - 1
            else:
                p, cnt = 0.002, m
            mean = p * cnt / m
            sigma = np.sqrt(cnt * p * (1 - p)) / m / np.sqrt(m)
            assert abs(rows[:, k].mean() - mean) < 5 * sigma, (b, k)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighted", [False, True])
def test_laplacian_matches_scipy_normalised_laplacian(seed, weighted):
    """Laplacian reading vs scipy: D^-1/2 A D^-1/2 = I - L_normed on nodes with
    positive degree (graphs without self-loops, since scipy ignores the
    diagonal of A)."""
    scipy_csgraph = pytest.importorskip("scipy.sparse.csgraph")
    n, s, K = 60 + 7 * seed, 200 + 30 * seed, 3 + seed
    edges = graphgen.random_graph(n, s, 300 + seed, self_loops=False)
    Y = graphgen.labels(n, K, 301 + seed, 0.2)
    w = graphgen.weights(s, 302 + seed) if weighted else None
    Z = oracle.embed(edges, Y, K, weights=w, laplacian=True)
    A = _pins.dense_adjacency(edges, n, w)
    L = scipy_csgraph.laplacian(A, normed=True)
    S = np.eye(n) - L
    deg = A.sum(axis=1)
    live = deg > 0
    S[~live, :] = 0.0
    expect = S @ _pins.dense_projection(Y, K)
    np.testing.assert_allclose(Z[live], expect[live], rtol=1e-12, atol=1e-14)
    assert np.all(Z[~live] == 0.0)


def test_round_counts_is_correct_rounding():
    rng = np.random.default_rng(5)
    C = rng.integers(0, 1 << 24, size=(400, 3), dtype=np.uint64)
    nk = rng.integers(1, 1 << 24, size=3, dtype=np.int64)
    # near-tie cases: quotients whose float32 rounding is hardest
    C[0] = [1, 3, 16777215]
    nk[:] = [3, 7, 16777213]
    Z = oracle.round_counts(C, nk)
    for u in range(C.shape[0]):
        for k in range(3):
            want = _pins.round_fraction_to_f32(Fraction(int(C[u, k]), int(nk[k])))
            assert Z[u, k] == want, (u, k)


def test_embed_rows_matches_dense():
    n, s, K = 400, 3000, 4
    edges, Y, w = _random_case(21, n, s, K, 0.1, True)
    rows = np.array([0, 5, 17, 399, 200, 5])
    r, Zr = oracle.embed_rows(edges, Y, K, rows, weights=w)
    Zd = _pins.dense_embedding(edges, Y, K, weights=w)
    assert np.array_equal(r, np.unique(rows))
    np.testing.assert_allclose(Zr, Zd[r], rtol=1e-12, atol=1e-14)
    edges_u, Yu, _ = _random_case(22, n, s, K, 0.1, False)
    r, Zr, Cr = oracle.embed_rows(edges_u, Yu, K, rows, with_counts=True)
    Zd = _pins.dense_embedding(edges_u, Yu, K)
    nk = np.bincount(Yu[Yu >= 0], minlength=K)
    np.testing.assert_allclose(Cr / np.maximum(nk, 1), Zd[r], rtol=1e-12, atol=1e-14)


def test_embed_rows_laplacian_matches_dense():
    scipy_csgraph = pytest.importorskip("scipy.sparse.csgraph")
    n, s, K = 120, 700, 3
    edges = graphgen.random_graph(n, s, 31, self_loops=False)
    Y = graphgen.labels(n, K, 32, 0.1)
    w = graphgen.weights(s, 33)
    rows = np.arange(0, n, 7)
    r, Zr = oracle.embed_rows(edges, Y, K, rows, weights=w, laplacian=True)
    A = _pins.dense_adjacency(edges, n, w)
    S = np.eye(n) - scipy_csgraph.laplacian(A, normed=True)
    S[A.sum(axis=1) == 0] = 0.0
    expect = (S @ _pins.dense_projection(Y, K))[r]
    np.testing.assert_allclose(Zr, expect, rtol=1e-12, atol=1e-14)


def test_error_codes():
    e = np.array([[0, 1]], np.int32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.embed(e, np.array([0, 2], np.int32), 2)
    assert ei.value.code == oracle.BAD_LABEL
    with pytest.raises(oracle.OracleError) as ei:
        oracle.embed(np.array([[0, 2]], np.int32), np.array([0, 1], np.int32), 2)
    assert ei.value.code == oracle.BAD_NODE
    with pytest.raises(oracle.OracleError) as ei:
        oracle.embed(e, np.array([0, -2], np.int32), 2)
    assert ei.value.code == oracle.BAD_LABEL
    with pytest.raises(oracle.OracleError) as ei:
        oracle.embed(e, np.array([0, 1], np.int32), 2,
                     weights=np.array([-1.0], np.float32), laplacian=True)
    assert ei.value.code == oracle.BAD_WEIGHT


# ---------------------------------------------------------------------------
# Unsupervised GEE: embedding alternated with k-means assignment steps
# ---------------------------------------------------------------------------
def _exact_round(edges, Y, K):
    """One round written out with exact rationals, independently of the
    oracle: integer counts by a loop over the edges, class means, squared
    distances; returns the new labels, per node the gap between the best
    and the second-best distance relative to the best (0 for ties), and the
    exact distances d[i][k] (None for empty classes)."""
    n = len(Y)
    C = [[0] * K for _ in range(n)]
    for u, v in edges:
        C[u][Y[v]] += 1
        C[v][Y[u]] += 1
    m = [sum(1 for y in Y if y == k) for k in range(K)]
    Z = [[Fraction(C[i][j], m[j]) if m[j] else Fraction(0) for j in range(K)]
         for i in range(n)]
    cen = [[Fraction(sum(C[i][j] for i in range(n) if Y[i] == k), m[k] * m[j])
            if m[k] and m[j] else Fraction(0) for j in range(K)] for k in range(K)]
    new, gaps, dist = [], [], []
    for i in range(n):
        row = [sum((Z[i][j] - cen[k][j]) ** 2 for j in range(K)) if m[k] else None
               for k in range(K)]
        d = sorted((row[k], k) for k in range(K) if m[k])
        new.append(d[0][1])
        gaps.append((d[1][0] - d[0][0]) / (d[0][0] + Fraction(1, 10**6))
                    if len(d) > 1 else Fraction(1))
        dist.append(row)
    return new, gaps, dist


@pytest.mark.parametrize("seed", range(6))
def test_unsupervised_round_matches_exact_rationals(seed):
    """One round (embed, then move every node to the nearest class mean)
    equals the exact-rational computation wherever the nearest mean is
    nearer than the next one by more than FP64 rounding can blur (gap above
    1e-9 of the distance), and the oracle's FP64 distances equal the exact
    ones to 1e-12 relative."""
    rng = np.random.default_rng(seed)
    n, K = 14, 3
    edges = graphgen.random_graph(n, 30, seed=100 + seed)
    Y0 = rng.integers(0, K, n).astype(np.int32)
    Y0[:K] = np.arange(K)  # every class present
    want, gaps, dist = _exact_round([tuple(e) for e in edges.tolist()], Y0.tolist(), K)
    got, rounds, moved = oracle.unsupervised(edges, Y0, K, max_iter=1)
    assert rounds == 1 and moved[0] == int(np.sum(got != Y0))
    clear = [i for i in range(n) if gaps[i] > Fraction(1, 10**9)]
    assert len(clear) >= n // 2
    assert [int(got[i]) for i in clear] == [want[i] for i in clear]
    nxt, D, T = oracle.unsup_round(edges, Y0, K)
    assert np.array_equal(nxt, got)
    for i in range(n):
        for k in range(K):
            if dist[i][k] is None:
                assert D[i, k] == 0.0
            else:
                assert abs(D[i, k] - float(dist[i][k])) <= 1e-12 * max(float(dist[i][k]), 1e-300)
                assert T[i, k] >= D[i, k]


def test_unsupervised_recovers_planted_blocks():
    """A planted partition with p_in/p_out = 50: the true blocks are a fixed
    point (one round, nothing moves); from 20% corrupted labels the loop
    returns to them; from random labels it finds them up to a relabelling;
    a class left empty by the start labels is never chosen."""
    import itertools
    n, K = 600, 3
    edges = graphgen.planted_edges(n, K, 6000, 50.0, seed=1)
    truth = graphgen.planted_labels(n, K)
    y, rounds, moved = oracle.unsupervised(edges, truth, K)
    assert rounds == 1 and moved == [0] and np.array_equal(y, truth)
    rng = np.random.default_rng(0)
    y0 = truth.copy()
    flip = rng.random(n) < 0.2
    y0[flip] = rng.integers(0, K, int(flip.sum()))
    y, rounds, moved = oracle.unsupervised(edges, y0, K)
    assert np.array_equal(y, truth) and moved[-1] == 0
    y, rounds, moved = oracle.unsupervised(edges, rng.integers(0, K, n).astype(np.int32), K)
    best = max(np.mean(np.array(p)[y] == truth) for p in itertools.permutations(range(K)))
    assert best == 1.0 and moved[-1] == 0
    y4, _, _ = oracle.unsupervised(edges, truth, K + 1)
    assert np.all(y4 < K)
    with pytest.raises(oracle.OracleError):
        oracle.unsupervised(edges, np.where(truth == 0, -1, truth).astype(np.int32), K)


def _pins_all_hold() -> bool:
    """Run a compact subset of the pins above; False if any fails."""
    try:
        for case in _pins.load_hand_cases():
            test_hand_cases(case)
        for seed in range(2):
            test_dense_closed_form(seed, True)
            test_dense_closed_form(seed, False)
        test_single_class_is_degree_over_n()
        for seed in range(2):
            test_laplacian_matches_scipy_normalised_laplacian(seed, True)
        for seed in range(3):
            test_unsupervised_round_matches_exact_rationals(seed)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", range(1, 10))
def test_pins_catch_planted_mistakes(mutation):
    """Each planted oracle mistake (dropped update, wrong index, transposed
    row, wrong class size, ...) must make at least one pin fail."""
    assert _pins_all_hold()
    oracle.set_mutation(mutation)
    try:
        assert not _pins_all_hold(), f"mutation {mutation} went unnoticed"
    finally:
        oracle.set_mutation(0)
    assert _pins_all_hold()
