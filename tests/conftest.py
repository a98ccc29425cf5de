"""Test configuration: the ``gpu`` marker and the repository root on sys.path.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything
else runs on the CPU (the oracle, its pins, host-side logic, and checks that
the library loads and exports every declared symbol).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libccmc")
    config.addinivalue_line("markers", "slow: long statistical run")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    return oracle.lib()
