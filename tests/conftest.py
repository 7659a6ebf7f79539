import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sphere_c1():
    """Rigid sphere a = 0.5, kD = 10, 320 curved quadratic triangles, N = 1920."""
    from paper_1311_5202_gb300 import inputs
    return inputs.icosphere(4, 0.5)
