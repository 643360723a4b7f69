import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpt.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def warm_weights():
    """The warm-start network, trained once per session the way the benchmark
    trains it (requested by GPU tests only)."""
    import bench
    w, info = bench.warm_start_weights(0)
    print("warm-start network:", {k: v for k, v in info.items() if k != "runs"}, info["runs"])
    return w
