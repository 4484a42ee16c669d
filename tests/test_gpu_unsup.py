"""gee_unsupervised through the C ABI against the FP64 oracle.

The paper fixes no precision for the clustering step (Section II only says Y
may come from clustering).  The oracle takes the assignment distances in
FP64; the library takes them in FP32, each difference, square and sum
rounded on its own.  So the two may choose different classes only where two
class means are nearly equally near, and by how much is bounded:

With z = RN32(C/m_j) and c = RN32(S/(m_k m_j)) (relative errors <= u = 2^-24
each), one term (z - c)^2 evaluated in FP32 differs from the exact term by
at most 5u(|z| + |c|)^2 (input errors 2u(|z|+|c|) in the difference, doubled
by squaring, one rounding of the square), and summing K terms in order adds
at most (K - 1)u times the sum of the terms.  So an FP32 distance is within
E(i,k) = (K + 4)u T(i,k) of the exact one, T(i,k) = sum_j (|z| + |c|)^2
(gee_oracle_unsup_round returns T).  The tests use (K + 5)u T with a 1 %
margin.  If the library picks class g for node i where the exact nearest
mean is b, then d(i,g) <= d(i,b) + E(i,g) + E(i,b): that is what every
round is checked against, from identical labels, and nodes whose nearest
mean leads by more than that slack must get exactly the oracle's class.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


def _slack(K, T):
    """Bound on the FP32 evaluation error of distances with scale T."""
    return 1.01 * (K + 5) * U32 * T


def _check_choice(edges, Y, K, got):
    """`got` (one assignment step from labels Y, on the GPU) against the
    oracle's FP64 round from the same labels; returns the number of nodes
    where they differ (all of them within the rounding slack)."""
    want, D, T = oracle.unsup_round(edges, Y, K)
    m = np.bincount(Y, minlength=K)
    assert np.all(m[got] > 0), "an empty class was chosen"
    i = np.arange(Y.size)
    slack = _slack(K, T[i, got]) + _slack(K, T[i, want])
    assert np.all(D[i, got] <= D[i, want] + slack)
    # nodes whose nearest mean leads every other class by more than the
    # largest slack any pair of classes can carry get exactly that class
    Dm = np.where(m[None, :] > 0, D, np.inf)
    best = Dm[i, want]
    second = np.partition(Dm, 1, axis=1)[:, 1] if K > 1 else np.full(Y.size, np.inf)
    decided = (second - best) > 2 * _slack(K, T.max(axis=1))
    assert np.array_equal(got[decided], want[decided])
    return int(np.sum(got != want))


def _purity(y, truth, K):
    return max(np.mean(np.array(p)[y] == truth) for p in itertools.permutations(range(K)))


@pytest.mark.parametrize("n,K,s,ratio,seed", [(20000, 8, 200000, 10.0, 1),
                                               (5000, 3, 30000, 4.0, 2),
                                               (3000, 17, 60000, 30.0, 3)])
def test_rounds_match_oracle_within_rounding(gee, n, K, s, ratio, seed):
    """Round by round from identical labels (the oracle's), the GPU's
    assignment is within the FP32 slack of the FP64 nearest mean, and its Z
    is the oracle's embedding of the labels it returns."""
    edges = graphgen.planted_edges(n, K, s, ratio, seed=seed)
    Y = np.random.default_rng(seed).integers(0, K, n).astype(np.int32)
    differ = 0
    with gee.Graph(_dev(edges), n) as g:
        for _ in range(6):
            y, Z, rounds, moved = g.unsupervised(_dev(Y), K, max_iter=1)
            got = y.cpu().numpy()
            assert rounds == 1 and moved == [int(np.sum(got != Y))]
            differ += _check_choice(edges, Y, K, got)
            assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, got, K))
            Y, _, _ = oracle.unsup_round(edges, Y, K)
    assert differ <= n // 1000 + 1


@pytest.mark.parametrize("n,K,s,ratio,seed", [(20000, 8, 200000, 10.0, 1),
                                               (3000, 17, 60000, 30.0, 3)])
def test_loop_reaches_a_fixed_point_of_the_oracle(gee, n, K, s, ratio, seed):
    """The full loop: where it stops (a round moved nothing), one FP64 oracle
    round from its labels moves no node beyond the rounding slack; its
    purity against the planted blocks matches the oracle's own loop."""
    edges = graphgen.planted_edges(n, K, s, ratio, seed=seed)
    truth = graphgen.planted_labels(n, K)
    rng = np.random.default_rng(seed)
    Y0 = truth.copy()
    flip = rng.random(n) < 0.3
    Y0[flip] = rng.integers(0, K, int(flip.sum()))
    want_y, want_rounds, _ = oracle.unsupervised(edges, Y0, K, max_iter=40)
    with gee.Graph(_dev(edges), n) as g:
        y, Z, rounds, moved = g.unsupervised(_dev(Y0), K, max_iter=40)
    y = y.cpu().numpy()
    assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, y, K))
    if rounds < 40:
        assert moved[-1] == 0
        _check_choice(edges, y, K, y)
    if K <= 8:
        assert _purity(y, truth, K) >= _purity(want_y, truth, K) - 0.01


def test_rmat_with_hub_rows_and_a_round_limit(gee):
    """Skewed degrees (hub rows in several chunks) and loops stopped by
    max_iter: every round within the slack, and the final Z is the
    embedding of the final labels."""
    n = 30000
    edges = graphgen.rmat_edges(15, n, 0, 400000, seed=8)
    K = 5
    Y0 = graphgen.labels(n, K, seed=9)
    with gee.Graph(_dev(edges), n) as g:
        y, Z, rounds, moved = g.unsupervised(_dev(Y0), K, max_iter=0)
        assert rounds == 0 and moved == []
        assert np.array_equal(y.cpu().numpy(), Y0)
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, Y0, K))
        Y = Y0
        for _ in range(3):
            y, Z, rounds, moved = g.unsupervised(_dev(Y), K, max_iter=1)
            got = y.cpu().numpy()
            _check_choice(edges, Y, K, got)
            assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, got, K))
            Y = got
        y, Z, rounds, moved = g.unsupervised(_dev(Y0), K, max_iter=3)
        assert rounds == 3 or moved[-1] == 0
        assert np.array_equal(Z.cpu().numpy(), oracle.embed_counts32(edges, y.cpu().numpy(), K))


def test_unsupervised_errors(gee):
    n = 500
    edges = graphgen.random_graph(n, 3000, seed=1)
    Y0 = graphgen.labels(n, 4, seed=2)
    with gee.Graph(_dev(edges), n) as g:
        bad = Y0.copy()
        bad[7] = -1
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(bad), 4)
        assert ei.value.name == "GEE_ERR_LABEL_RANGE"
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(Y0), 65)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"
    w = graphgen.weights(3000, seed=3)
    with gee.Graph(_dev(edges), n, weights=_dev(w)) as g:
        with pytest.raises(gee.GeeError) as ei:
            g.unsupervised(_dev(Y0), 4)
        assert ei.value.name == "GEE_ERR_UNSUPPORTED"


def test_rows_of_2_23_arcs_are_refused(gee):
    """The assignment recovers the exact counts from Z as rint(Z * m_j),
    exact only for counts below 2^23: a graph with a row of 2^23 arcs (a
    star) is refused with GEE_ERR_OVERFLOW before any round runs; one arc
    fewer runs."""
    import torch
    for leaves, ok in ((1 << 23, False), ((1 << 23) - 1, True)):
        n = leaves + 1
        e = torch.zeros((leaves, 2), dtype=torch.int32, device="cuda")
        e[:, 1] = torch.arange(1, n, dtype=torch.int32, device="cuda")
        Y0 = torch.zeros(n, dtype=torch.int32, device="cuda")
        Y0[1::2] = 1
        with gee.Graph(e, n) as g:
            if ok:
                y, Z, rounds, moved = g.unsupervised(Y0, 2, max_iter=1)
                assert rounds == 1
            else:
                with pytest.raises(gee.GeeError) as ei:
                    g.unsupervised(Y0, 2, max_iter=1)
                assert ei.value.name == "GEE_ERR_OVERFLOW"
        del e, Y0
        torch.cuda.empty_cache()
