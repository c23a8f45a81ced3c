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


def test_sm103a_only_build_flags():
    # the library is compiled and linked for sm_103a alone: one -gencode, no PTX for other targets
    from paper_2402_10914_gb300 import build
    gencodes = [build.ARCH[i + 1] for i, a in enumerate(build.ARCH) if a == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert all("-arch" not in f and "compute_" not in f for f in build.flags() if f not in build.ARCH)


def test_noalloc_refuses_what_create_refuses_before_device_work(libpath):
    # dfgks_residual_noalloc validates its configuration before touching the device, so these
    # refusals need no GPU; the pointers are never dereferenced
    import ctypes
    from paper_2402_10914_gb300 import _lib
    L = _lib.lib()
    buf = (ctypes.c_double * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)

    def call(nx, ny, bc):
        cfg = _lib.Config()
        assert L.dfgks_config_default(ctypes.byref(cfg), nx, ny) == 0
        cfg.bc_xlo, cfg.bc_xhi, cfg.bc_ylo, cfg.bc_yhi = bc
        h = ctypes.c_void_p()
        created = L.dfgks_create(ctypes.byref(cfg), None, ctypes.byref(h)) if nx * ny <= 16 else None
        rc = L.dfgks_residual_noalloc(ctypes.byref(cfg), None, p, p, ctypes.c_double(1e-3), 0, p, p, p, p)
        return rc, created

    REF, OUT, PER = 2, 1, 0
    # a walled or periodic direction needs 3 cells (its ghost map copies or mirrors 3 cells)
    for nx, ny, bc in [(2, 5, (REF, REF, OUT, OUT)), (2, 5, (REF, OUT, OUT, OUT)), (5, 2, (OUT, OUT, PER, PER)),
                       (2, 5, (PER, PER, OUT, OUT)), (5, 2, (OUT, OUT, OUT, REF))]:
        rc, created = call(nx, ny, bc)
        assert rc == _lib.EINVAL, (nx, ny, bc)
        assert created == _lib.EINVAL, (nx, ny, bc)
    # a side above 128 cells is refused, also when the cell count is small (1024 x 16)
    for nx, ny in [(129, 128), (1024, 16), (16, 129)]:
        rc, _ = call(nx, ny, (OUT, OUT, OUT, OUT))
        assert rc == _lib.EINVAL, (nx, ny)


def test_ctypes_structs_match_the_header(tmp_path):
    # the binding's Config / Counters layouts against the C compiler's view of include/dfgks.h
    import ctypes
    from paper_2402_10914_gb300 import _lib
    fields = [f for f, _ in _lib.Config._fields_]
    cfields = [f for f, _ in _lib.Counters._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dfgks.h"', 'int main(void) {',
             '  printf("config %zu\\n", sizeof(dfgks_config));', '  printf("counters %zu\\n", sizeof(dfgks_counters));']
    lines += ['  printf("%s %%zu\\n", offsetof(dfgks_config, %s));' % (f, f) for f in fields]
    lines += ['  printf("c.%s %%zu\\n", offsetof(dfgks_counters, %s));' % (f, f) for f in cfields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    assert int(out["config"]) == ctypes.sizeof(_lib.Config)
    assert int(out["counters"]) == ctypes.sizeof(_lib.Counters)
    for f in fields:
        assert int(out[f]) == getattr(_lib.Config, f).offset, f
    for f in cfields:
        assert int(out["c." + f]) == getattr(_lib.Counters, f).offset, f


INVALID = {
    "nx_zero": dict(nx=0), "ny_negative": dict(ny=-4), "nx_above_2^20": dict(nx=(1 << 20) + 1),
    "cells_above_2^28": dict(nx=1 << 15, ny=(1 << 13) + 1), "empty_domain": dict(x1=0.0),
    "gamma_one": dict(gamma=1.0), "cfl_zero": dict(cfl=0.0), "eps_zero": dict(eps=0.0), "dH_zero": dict(dH=0.0),
    "dL_above_one": dict(dL=1.5), "C2_negative": dict(C2=-1.0), "bc_unknown": dict(bc_yhi=3),
    "periodic_one_side": dict(bc_xlo=0), "periodic_two_cells": dict(nx=2, bc_xlo=0, bc_xhi=0),
    "wall_two_cells": dict(ny=2, bc_ylo=2), "tau_reading_2": dict(tau_reading=2), "time_scheme_5": dict(time_scheme=5),
    "dt_rule_2": dict(dt_rule=2), "df_states_2": dict(df_states=2), "alpha_source_2": dict(alpha_source=2),
}


def test_batch_and_decomposition_refuse_alpha_from_the_new_state(libpath):
    # alpha_source = 1 is built for the single-problem handle only: the batch and the block
    # decomposition refuse it with EINVAL before any CUDA call (so this runs without a GPU)
    import ctypes
    from paper_2402_10914_gb300 import _lib
    L = _lib.lib()
    cfg = _lib.Config()
    assert L.dfgks_config_default(ctypes.byref(cfg), 16, 16) == 0
    cfg.alpha_source = 1
    cfgs = (_lib.Config * 1)(cfg)
    flux = (ctypes.c_int * 1)(0)
    b = ctypes.c_void_p(1234)
    assert L.dfgks_batch_create(ctypes.cast(cfgs, ctypes.c_void_p), ctypes.cast(flux, ctypes.c_void_p), 1, None,
                                ctypes.byref(b)) == _lib.EINVAL
    assert b.value is None
    d = ctypes.c_void_p(1234)
    assert L.dfgks_decomp_create(ctypes.byref(cfg), 2, 1, None, ctypes.byref(d)) == _lib.EINVAL
    assert d.value is None


@pytest.mark.parametrize("name", list(INVALID))
def test_create_refuses_invalid_configs_before_device_work(libpath, name):
    # dfgks_create and dfgks_batch_create validate the whole configuration before any CUDA call,
    # so this runs without a GPU
    import ctypes
    from paper_2402_10914_gb300 import _lib
    L = _lib.lib()
    cfg = _lib.Config()
    assert L.dfgks_config_default(ctypes.byref(cfg), 16, 12) == 0
    for k, v in INVALID[name].items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p(1234)
    assert L.dfgks_create(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.EINVAL
    assert h.value is None                                   # *out cleared on failure
    cfgs = (_lib.Config * 2)()
    assert L.dfgks_config_default(ctypes.byref(cfgs[0]), 16, 16) == 0
    cfgs[1] = cfg
    flux = (ctypes.c_int * 2)(0, 1)
    b = ctypes.c_void_p(1234)
    assert L.dfgks_batch_create(ctypes.cast(cfgs, ctypes.c_void_p), ctypes.cast(flux, ctypes.c_void_p), 2, None,
                                ctypes.byref(b)) == _lib.EINVAL
    assert b.value is None
