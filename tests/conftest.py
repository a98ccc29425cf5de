"""Test configuration: the ``gpu`` marker, the repository root on sys.path, and
an up-to-date build of the oracle and of libccmc before any test runs.

Tests marked ``gpu`` need a CUDA device and call the library through its C ABI;
everything else runs on the CPU (the oracle and its pins, host-side logic, and
checks that the library loads and exports every declared symbol).
"""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libccmc")


def pytest_sessionstart(session):
    from oracle import build as oracle_build

    oracle_build.build()
    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        from paper_2301_11735_gb300 import build as lib_build

        lib_build.build()


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    return oracle.lib()
