import os
import sys

# one BLAS thread: the oracle's matrices are small, and many idle BLAS threads
# on a large host slow them down by orders of magnitude
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest  # noqa: E402

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
