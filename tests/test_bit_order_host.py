"""The integer-order helpers the sweep kernels use for maxima, minima and tests of non-negative
values (tests/bit_order_check.cu), built for the host: the same bits as fmax / fmin and the same
decisions as < on non-negative values, and a range test that rejects negatives, -0 and NaN."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2402_10914_gb300", "csrc")


def test_bit_order_helpers_match_floating_point(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "bit_order_check")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(HERE, "bit_order_check.cu"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("0 mismatches")
