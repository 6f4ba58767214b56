import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cfg1():
    """N=128 gapped random-spectrum problem: 64 occupied eigenvalues U[-1,-0.2],
    64 empty U[0.2,1], Haar eigenvectors, A and 8 H1_k symmetric N(0, 1/N)."""
    import workloads
    return workloads.random_spectrum(128, nocc=64, k=8, seed=0)
