"""pytest configuration: the `gpu` marker and shared fixtures.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything
else runs on a CPU-only host (the oracle, its pins, host-side logic, and the
check that the C-ABI library exports every declared symbol).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
