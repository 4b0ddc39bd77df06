"""Shared test set-up: the repository root on sys.path and the `gpu` marker.

Tests marked `gpu` need a CUDA GPU and the built library; everything else runs on a CPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and libsnect.so")


@pytest.fixture(scope="session")
def gpu_lib():
    """Builds (if needed) and loads libsnect.so; skips nothing: a GPU test without a GPU fails."""
    import torch

    import paper_1711_08095_gb300 as snect

    if not torch.cuda.is_available():
        pytest.fail("gpu test collected on a machine without a CUDA GPU")
    lib = snect.load(build_if_missing=True)
    torch.cuda.init()
    return lib
