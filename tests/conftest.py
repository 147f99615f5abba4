import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def params():
    from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table
    return synthetic_gfn1_table()


@pytest.fixture(scope="session")
def water64():
    from paper_2606_28022_b300.inputs.geometry import water_cluster
    return water_cluster(64, 1)
