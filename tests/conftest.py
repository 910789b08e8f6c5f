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


# The GPU suite runs under an outer time limit on the GPU machines.  Should it ever run long
# (a slow host, a busy GPU), the GPU tests that would start after this many seconds are skipped
# with a message, so that the run reports what it checked instead of being killed mid-test.
_GPU_SUITE_BUDGET_S = float(os.environ.get("ED_GPU_SUITE_BUDGET_S", "1000"))
_T_START = None


def pytest_sessionstart(session):
    global _T_START
    import time

    _T_START = time.monotonic()


def pytest_runtest_setup(item):
    if _T_START is None or item.get_closest_marker("gpu") is None:
        return
    import time

    spent = time.monotonic() - _T_START
    if spent > _GPU_SUITE_BUDGET_S:
        pytest.skip("GPU suite time budget (%.0f s) spent after %.0f s" % (_GPU_SUITE_BUDGET_S, spent))
