import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def net32():
    from paper_2511_10558_gb300 import synth
    return synth.make_network(32, 200)


@pytest.fixture(scope="session")
def net150():
    from paper_2511_10558_gb300 import synth
    return synth.make_network(150, 1500)
