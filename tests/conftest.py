import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built renderer library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny_workload():
    import scenegen
    return scenegen.tiny()


@pytest.fixture(scope="session")
def tiny_arrays(tiny_workload):
    import scenegen
    w = tiny_workload
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    return sig, uvw, beta
