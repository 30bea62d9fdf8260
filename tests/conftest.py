import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


def uniform_system(N, L, seed):
    """Neutral +-1 charges at uniform positions in the centred box."""
    from paper_2412_04595_gb300 import workloads
    return workloads.uniform_neutral(N, L, seed)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build_oracle()
    from oracle import sog
    return sog
