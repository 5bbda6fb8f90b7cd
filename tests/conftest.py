import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs longer than a few seconds")


@pytest.fixture(scope="session")
def small_problem():
    from paper_2411_09244_gb300.inputs import config_small
    return config_small(n_f=16, nc=4, J=2, ell=1, N=4, P=8)
