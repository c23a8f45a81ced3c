"""Build the CUDA library libdfgks.so in place (sm_103a only).

Both translation units are compiled in parallel with one ``-gencode`` and linked into
``paper_2402_10914_gb300/libdfgks.so``.  No torch extension machinery: the library has a plain
C ABI (``include/dfgks.h``) and is loaded with ctypes.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdfgks.so")
SOURCES = ["dfgks_kernels.cu", "dfgks_capi.cu", "dfgks_probe.cu", "dfgks_noalloc.cu", "dfgks_batch.cu", "dfgks_adjoint.cu",
           "dfgks_decomp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


# the sources that define the single-problem forward kernels (the profiled ones)
FORWARD_KERNEL_SOURCES = ["dfgks_device.cuh", "dfgks_bodies.cuh", "dfgks_kernels.cu", "dfgks_internal.h"]


def kernel_source_hash() -> str:
    """sha256 (first 16 hex digits) over the forward kernels' sources and the compile flags: a
    profile summary records it, and counts measured on other sources are not used."""
    import hashlib
    h = hashlib.sha256()
    for f in FORWARD_KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + ["-O3", "-std=c++17"]).encode())
    return h.hexdigest()[:16]


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "dfgks.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *flags(extra), "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
