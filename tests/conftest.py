import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgee.so")
    config.addinivalue_line(
        "markers", "slow: full-size workloads (minutes on the host side)")


@pytest.fixture(scope="session")
def tiny_sbm_graph():
    """The 5-block SBM (5 x 2000 nodes, p_in 0.02, p_out 0.002), seed 1."""
    import graphgen
    return graphgen.tiny_sbm(seed=1)
