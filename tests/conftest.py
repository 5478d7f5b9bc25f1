"""Shared pytest configuration: the ``gpu`` marker and the oracle build."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librlb.so")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
