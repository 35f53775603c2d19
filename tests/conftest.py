import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def laplacian_2d_eigs(m: int) -> np.ndarray:
    """Closed-form spectrum of the m x m 5-point Dirichlet Laplacian, ascending."""
    c = 2.0 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
    return np.sort(((4.0 - c)[:, None] - c[None, :]).ravel())


def laplacian_3d_eigs(m: int) -> np.ndarray:
    """Closed-form spectrum of the m^3 7-point Dirichlet Laplacian, ascending."""
    c = 2.0 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
    return np.sort(((6.0 - c)[:, None, None] - c[None, :, None] - c[None, None, :]).ravel())


@pytest.fixture(scope="session")
def lap2d_eigs():
    return laplacian_2d_eigs


@pytest.fixture(scope="session")
def lap3d_eigs():
    return laplacian_3d_eigs
