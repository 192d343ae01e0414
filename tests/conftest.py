import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session", autouse=True)
def oracle_threads():
    """The oracle's projector loops on every host core (its results do not
    depend on the thread count)."""
    from oracle import siddon
    siddon.set_threads(os.cpu_count() or 1)


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import siddon
    return siddon.lib()
