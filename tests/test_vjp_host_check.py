"""Builds tests/vjp_host_check.cu as a host program (the reverse products of the GPU adjoint and the
forward device functions they differentiate, compiled for the CPU from the same headers) and runs
it: every reverse product must match central finite differences of its forward function."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2402_10914_gb300", "csrc")


def test_reverse_products_match_finite_differences(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "vjp_host_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(HERE, "vjp_host_check.cu"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert r.stdout.count(" ok") >= 10
