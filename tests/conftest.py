"""Shared pytest configuration: the `gpu` marker and session fixtures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The product library bound to cuda:0. GPU tests fail (not skip) without a GPU."""
    import paper_1312_3018_gb300 as pkg
    assert cuda_available(), "GPU test requested but no CUDA device is visible"
    return pkg
