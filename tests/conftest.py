import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libqdta.so")


@pytest.fixture(scope="session")
def small_instance():
    from paper_2104_12911_gb300 import synth
    return synth.config_small(0)
