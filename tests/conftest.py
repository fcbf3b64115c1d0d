"""Shared pytest setup: repository root on sys.path, GPU gating, common fixtures."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmpgpu.so")


@pytest.fixture(scope="session")
def oracle():
    from oracle import mpref

    mpref.build()
    return mpref


@pytest.fixture(scope="session")
def mp():
    """The CUDA library binding; requires a GPU (tests using it are marked gpu)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_14926_gb300 as mpg

    mpg.load()  # raises if libmpgpu.so is missing: no silent fallback
    return mpg
