import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def sv_grid4x6():
    """State vector of the 24-qubit, 14-cycle 4x6 workload (FP64 oracle O1)."""
    import workloads as W
    from oracle import statevector as sv
    w = W.workload("grid4x6_d14")
    return w, sv.simulate(w.circuit)
