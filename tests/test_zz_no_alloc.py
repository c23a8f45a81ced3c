"""The allocation-free stage operator (dfgks_residual_noalloc) against the handle-based one.

Callers that cannot allocate device memory (graph construction, pool-managed hosts, latency-bound
loops) use dfgks_residual_noalloc, whose intermediates live in a fixed device array instead of
buffers allocated by dfgks_create.  Its results must equal those of dfgks_residual.  The file is
named to be collected last; the test also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2402_10914_gb300 import inputs as I
from tests.parity_util import comp_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(settings, W, alpha, dt, flux):
    from paper_2402_10914_gb300 import _lib
    from paper_2402_10914_gb300.solver import make_config
    cfg = make_config(settings)
    L = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    dL, dLt = torch.empty_like(L), torch.empty_like(L)
    an = torch.empty(W.shape[1:], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = _lib.lib().dfgks_residual_noalloc(C.byref(cfg), C.c_void_p(stream), p(W), p(alpha), float(dt), int(flux),
                                            p(L), p(dL), p(dLt), p(an))
    return rc, (L, dL, dLt, an)


def test_noalloc_stage_operator_matches_handle_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_10914_gb300 import _lib
    from paper_2402_10914_gb300.solver import Solver
    cases = [I.quadrants(96, seed=3), I.random_rough(23, 17, seed=6, bc=(I.PERIODIC, I.PERIODIC, I.REFLECT, I.OUTFLOW),
                                                     flux=I.LF, time_limiter=0)]
    for w in cases:                          # two calls in a row, different meshes and fluxes
        s = w.settings
        W = torch.as_tensor(w.W0, dtype=torch.float64, device="cuda").contiguous()
        alpha = torch.as_tensor(np.random.default_rng(1).uniform(0.2, 1.0, (s.ny, s.nx)), device="cuda").contiguous()
        dt = 1e-3
        rc, got = _noalloc(s, W, alpha, dt, s.flux)
        assert rc == _lib.OK, _lib.status_string(rc)
        with Solver(s) as sol:
            ref = sol.residual(W, alpha, dt, flux=s.flux)
        torch.cuda.synchronize()
        for g, r in zip(got[:3], ref[:3]):
            assert comp_rel_err(g.cpu().numpy(), r.cpu().numpy()) <= 1e-12
        assert comp_rel_err(got[3].cpu().numpy()[None], ref[3].cpu().numpy()[None], floor_frac=1e-12) <= 1e-12
    # refused before any device work: a side above 128 cells (also at a small cell count), and a
    # walled direction with fewer than 3 cells, which dfgks_create refuses as well
    for nx, ny, bc in [(129, 128, (I.OUTFLOW,) * 4), (1024, 16, (I.OUTFLOW,) * 4),
                       (2, 5, (I.REFLECT, I.REFLECT, I.OUTFLOW, I.OUTFLOW))]:
        bad = I.Settings(nx=nx, ny=ny, bc=bc)
        Wb = torch.ones((4, ny, nx), dtype=torch.float64, device="cuda")
        ab = torch.ones((ny, nx), dtype=torch.float64, device="cuda")
        rc, _ = _noalloc(bad, Wb, ab, 1e-3, I.GKS)
        assert rc == _lib.EINVAL, (nx, ny, bc)
