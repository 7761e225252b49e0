import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU physics runs of the oracle")


@pytest.fixture(scope="session", autouse=True)
def _oracle_threads():
    # The oracle is deterministic for any thread count; use the host's cores.
    try:
        import oracle
        oracle.set_threads(min(os.cpu_count() or 1, 16))
    except Exception:
        pass
    yield
