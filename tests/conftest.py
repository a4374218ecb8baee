"""Shared test set-up: the ``gpu`` marker and the repository root on sys.path.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything
else runs on the CPU only (the oracle, host logic, ABI exports, gloo ranks).
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
def orc():
    import oracle
    oracle.build()
    return oracle
