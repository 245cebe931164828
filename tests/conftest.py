"""Shared pytest configuration.

Marker ``gpu``: the test needs a CUDA device and the compiled library.
Everything else runs on the CPU (oracle pins, host logic, the C-ABI symbol
check and the multi-rank exchange algebra over gloo).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libsurvgpu.so")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def lib():
    """The loaded CUDA library (gpu tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08183_gb300 import binding
    return binding.load()
