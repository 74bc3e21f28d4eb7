import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1810_07026_gb300 import inputs  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def params():
    return inputs.make_params(0)


@pytest.fixture(scope="session")
def param_text(params):
    return inputs.params_text(params)


@pytest.fixture(scope="session")
def oracle(param_text):
    from oracle.oracle import Oracle
    return Oracle(param_text)


def box_of(L):
    return np.array([L, L, L], dtype=np.float64)
