import os
import sys

# The oracle's Lanczos recursions work on vectors of 1e3 - 1e7 elements one level at a time; a
# multi-threaded BLAS spends more time waking its threads than computing on them (measured: a
# 15,876-state continued fraction runs about 60x faster on one thread).  Set before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libed.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")
