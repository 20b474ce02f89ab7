import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


@pytest.fixture(scope="session", autouse=True)
def _oracle_threads():
    """The oracle's line loops use every host core (its results do not depend on
    the thread count)."""
    import oracle
    oracle.set_threads(min(os.cpu_count() or 1, 32))
    yield
