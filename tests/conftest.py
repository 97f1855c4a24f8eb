import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test (full-size oracle build)")


@pytest.fixture(scope="session")
def sphere_small():
    """PEC sphere radius 0.3 wavelengths, icosphere with 1,280 triangles
    (1,920 RWG unknowns), wavelength 1."""
    from synth import icosphere
    from oracle.rwg import RWGMesh
    xyz, tri = icosphere(3, 0.3)
    return RWGMesh(xyz, tri)


@pytest.fixture(scope="session")
def sphere_tiny():
    """PEC sphere radius 0.15 wavelengths, 320 triangles (480 unknowns)."""
    from synth import icosphere
    from oracle.rwg import RWGMesh
    xyz, tri = icosphere(2, 0.15)
    return RWGMesh(xyz, tri)


@pytest.fixture(scope="session")
def dense_small(sphere_small):
    return sphere_small.dense()
