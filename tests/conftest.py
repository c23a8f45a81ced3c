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


@pytest.fixture(scope="session", autouse=True)
def _cuda_library_built():
    """Tests load libdfgks.so (ABI exports, host-side block plans, the GPU paths): compile it once per
    session when it is missing or older than its sources, as __graft_entry__.build() does (nvcc
    cross-compiles without a GPU).  The library itself never builds on demand: a product call
    without it raises."""
    from paper_2402_10914_gb300 import build as cuda_build
    cuda_build.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
