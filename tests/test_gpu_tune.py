"""gee_autotune on the GPU: every grid point of the table holds the fastest
of the strategies it timed, and GEE_AUTO then follows the table while the
results stay those of the oracle."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gee():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_04403_gb300 as gee
    gee.load()
    yield gee
    gee.tune_set([])


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_autotune_table_and_auto_results(gee):
    table = gee.autotune(0)
    assert len(table) == 8 * 4
    for c in table:
        times = {"atomic": c["ms_atomic"], "private": c["ms_private"],
                 "segmented": c["ms_segmented"]}
        measured = {k: v for k, v in times.items() if v >= 0}
        assert "atomic" in measured and "segmented" in measured
        assert (c["log2_cells"] <= 15) == ("private" in measured)
        assert c["strategy"] in measured
        # the choice is the fastest strategy (its time is the minimum,
        # atomic's recorded time being its best block size)
        assert measured[c["strategy"]] <= min(measured.values()) + 1e-6
    # GEE_AUTO follows the table; results are the oracle's
    for (n, s, K) in [(300, 5000, 7), (20000, 30000, 12), (5000, 400000, 3)]:
        e = graphgen.random_graph(n, s, seed=n)
        Y = graphgen.labels(n, K, seed=s, frac_unlabeled=0.1)
        lc, ld = np.log2(n * K), np.log2(max(2 * s / (n * K), 1 / 1024))
        near = min(table, key=lambda c: abs(c["log2_cells"] - lc) + abs(c["log2_density"] - ld))
        want_strategy = near["strategy"]
        if want_strategy == "private" and n * K > 220 * 1024 // 4:
            want_strategy = "atomic"
        assert gee.pick_strategy(s, n, K) == want_strategy
        got = gee.embed(_dev(e), _dev(Y), K).cpu().numpy()
        assert np.array_equal(got, oracle.embed_counts32(e, Y, K))
    gee.tune_set([])
    assert gee.tune_table() == []
