import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the oracle's OpenMP threads sleep between parallel regions instead of spinning: many tests run it
# on small meshes with thousands of short regions, where spinning threads compete with each other
# and with whatever else runs on the host (set before the oracle library loads its runtime)
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
