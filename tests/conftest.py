import os
import sys

# single-threaded BLAS: the oracle's Algorithm 2 trajectory depends on rounding, and threaded
# reductions would make it differ from run to run
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
