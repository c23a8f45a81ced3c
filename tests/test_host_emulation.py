"""The CUDA path's per-thread bodies built for the host (tests/host_emulation.cu): the stage
operator and its reverse sweep, run body by body as the kernels call them, against the oracle's
stage operator and its tape adjoint.  Built under AddressSanitizer where the toolchain has it, so an
out-of-bounds index in the bodies fails here, on the CPU."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
from paper_2402_10914_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2402_10914_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("emu")
    exe = str(d / "host_emulation")
    base = [nvcc, "-O1", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
            os.path.join(HERE, "host_emulation.cu"), "-o", exe]
    asan = ["-Xcompiler", "-fsanitize=address,-fno-omit-frame-pointer", "-Xlinker", "-lasan"]
    if subprocess.run(base + asan, capture_output=True).returncode != 0:
        subprocess.run(base, check=True, capture_output=True)

    def run(s, W, alpha, dt, Lb, dLb, dLtb):
        hdr = struct.pack("10i", s.nx, s.ny, *s.bc, s.flux, s.time_limiter, s.tau_reading, s.gp_fallback)
        hdr += struct.pack("12d", s.x0, s.x1, s.y0, s.y1, s.gamma, s.alpha_thres, s.dH, s.dL, s.eps, s.C1, s.C2, dt)
        fin, fout = str(d / "in.bin"), str(d / "out.bin")
        with open(fin, "wb") as f:
            f.write(hdr)
            for a in (W, alpha, Lb, dLb, dLtb):
                f.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0"))
        assert r.returncode == 0, r.stderr[-2000:]
        return np.fromfile(fout).reshape(5, 4, s.ny, s.nx)
    return run


def rel(a, b, floor=1e-300):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


CASES = [
    ("lf_smooth_periodic", lambda: I.random_smooth(9, 8, seed=21, amp=0.08, flux=I.LF, time_limiter=0), "rand"),
    ("gks_smooth_outflow_limiter", lambda: I.random_smooth(9, 8, seed=22, amp=0.08, bc=(I.OUTFLOW,) * 4,
                                                           flux=I.GKS, time_limiter=1), "rand"),
    ("gks_smooth_reflect", lambda: I.random_smooth(10, 7, seed=23, amp=0.08, bc=(I.REFLECT,) * 4, flux=I.GKS,
                                                   time_limiter=1), "ones"),
    ("gks_tau_n", lambda: I.random_smooth(8, 9, seed=24, flux=I.GKS, time_limiter=0, tau_reading=1), "ones"),
    ("gks_rough_limiter", lambda: I.random_rough(14, 11, seed=41, flux=I.GKS, time_limiter=1), "rand"),
    ("lf_rough_periodic", lambda: I.random_rough(14, 11, seed=44, bc=(I.PERIODIC,) * 4, flux=I.LF,
                                                 time_limiter=0), "rand"),
    ("quadrants", lambda: I.quadrants(24, seed=2), "ones"),
    # degenerate meshes: one cell, one row, one column, the smallest periodic and walled meshes
    ("gks_one_cell", lambda: I.random_rough(1, 1, seed=5, flux=I.GKS, time_limiter=1), "rand"),
    ("lf_one_row", lambda: I.random_rough(7, 1, seed=6, flux=I.LF, time_limiter=0), "rand"),
    ("gks_one_column", lambda: I.random_rough(1, 7, seed=5, flux=I.GKS, time_limiter=1), "rand"),
    ("gks_3x3_periodic", lambda: I.random_rough(3, 3, seed=5, bc=(I.PERIODIC,) * 4, flux=I.GKS,
                                                time_limiter=1), "rand"),
    ("gks_3x5_reflect", lambda: I.random_smooth(3, 5, seed=7, bc=(I.REFLECT,) * 4, flux=I.GKS,
                                                time_limiter=1), "ones"),
]


@pytest.mark.parametrize("name,make,akind", CASES, ids=[c[0] for c in CASES])
def test_host_build_matches_oracle(emu, name, make, akind):
    w = make()
    s = w.settings
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0.0, 1.0, (s.ny, s.nx)) if akind == "rand" else np.ones((s.ny, s.nx))
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    Lb, dLb, dLtb = (rng.normal(size=w.W0.shape) for _ in range(3))
    out = emu(s, w.W0, alpha, dt, Lb, dLb, dLtb)
    L, dL, dLt, _, _ = oracle.residual(s, w.W0, alpha, dt)
    # the limited dL/dt carries the limiter weight, a near-switch on discontinuous data: rounding
    # differences in the smoothness indicators move it by up to ~3e-8 there
    assert rel(out[0], L) <= 1e-12 and rel(out[1], dL) <= 1e-11 and rel(out[2], dLt) <= 1e-7
    ref = oracle.residual_vjp(s, w.W0, alpha, dt, Lb, dLb, dLtb)
    # floor 1: the cotangents are N(0, 1); on one cell with outflow ghosts the state is uniform
    # for every W, L is identically zero and both sides return rounding noise (~1e-16)
    assert rel(out[3], ref, 1.0) <= 1e-12, rel(out[3], ref, 1.0)
    assert rel(out[4], ref, 1.0) <= 1e-12, rel(out[4], ref, 1.0)     # GKS reverse from the forward's tape
