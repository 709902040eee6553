import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libfpp.so")
    config.addinivalue_line("markers", "slow: long-running CPU case")


@pytest.fixture(scope="session")
def tiny_data():
    import workloads as W
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    return w, X, Q


@pytest.fixture(scope="session")
def tiny_index(tiny_data):
    import oracle as O
    w, X, Q = tiny_data
    return O.build_index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
