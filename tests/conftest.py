import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


_ORACLES = {}


@pytest.fixture(scope="session")
def oracle_for():
    """Cached oracle instances keyed by (n, jitter, seed, affine)."""
    from oracle import Oracle
    from paper_1811_03339_gb300 import inputs

    def get(n, jitter=0.0, seed=0, affine=None):
        key = (n, jitter, seed, None if affine is None else tuple(map(tuple, affine)))
        if key not in _ORACLES:
            mesh = inputs.cube_mesh(n, jitter, seed, affine)
            _ORACLES[key] = (mesh, Oracle.from_mesh(mesh))
        return _ORACLES[key]

    return get
