"""pytest configuration: the ``gpu`` marker and shared helpers.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything
else (the oracle against its pins, the input generator, host logic, loading
the C-ABI library and checking its exports) runs on a CPU-only host.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libfbp.so")
    config.addinivalue_line("markers", "slow: long-running (still part of the default run)")
