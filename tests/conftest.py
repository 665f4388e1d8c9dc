import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: CPU test that runs the oracle for tens of seconds")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.core.lib()  # builds the oracle if needed
    return oracle
