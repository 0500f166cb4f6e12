"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the built GB300 library; the rest
run on any CPU host (the oracle is compiled with gcc on first use).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpulib():
    """The compiled CUDA library, loaded; fails loudly when it is missing."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01850_gb300 import gmres as G
    return G.lib()
