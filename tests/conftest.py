"""Test configuration: the ``gpu`` marker and shared fixtures.

``-m "not gpu"`` runs on any machine (oracle pins, host logic, symbol checks);
``-m gpu`` needs a GB300 and calls the CUDA library through its C-ABI.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled GPSS library")


@pytest.fixture(scope="session")
def gpss():
    """The CUDA library's Python binding (built on first use)."""
    from paper_2603_00280_gb300 import gpss as g
    g.load()
    return g
