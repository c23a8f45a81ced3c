"""CPU-side checks of the C-ABI library: it builds, loads, and exports every declared entry point."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"DFGKS_API\s+[\w\s\*]+?\b(dfgks_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_10914_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("dfgks_create", "dfgks_destroy", "dfgks_set_ic", "dfgks_step", "dfgks_residual",
                     "dfgks_adjoint_residual", "dfgks_get_state"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(dfgks_\w+)", out))
    missing = declared_symbols() - exported
    assert not missing, missing


def test_library_loads_and_binds_without_gpu(libpath):
    import ctypes
    from paper_2402_10914_gb300 import _lib
    L = _lib.lib()
    for name in declared_symbols():
        assert hasattr(L, name)
    assert set(_lib.exported_symbols()) == declared_symbols()
    assert _lib.status_string(_lib.ENONPOS).startswith("positivity")
    # argument validation happens before any device work
    cfg = _lib.Config()
    assert L.dfgks_config_default(ctypes.byref(cfg), 16, 8) == 0
    assert cfg.alpha_thres == 0.5 and cfg.dH == 0.85 and cfg.C2 == 5.0
    cfg.nx = 0
    h = ctypes.c_void_p()
    assert L.dfgks_create(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.EINVAL
    assert L.dfgks_destroy(None) == 0


def test_sm103a_cubin_only(libpath):
    # the library carries sm_103a code only (no PTX for other architectures)
    r = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    elfs = [l for l in r.stdout.splitlines() if ".cubin" in l]
    assert elfs and all("sm_103a" in l for l in elfs), r.stdout
