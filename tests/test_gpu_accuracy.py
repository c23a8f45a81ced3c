"""The paper's accuracy tables (Sect. 4.1) reproduced on the CUDA path, mesh by mesh: the density
error norms of the smooth sine wave after one period against the printed Tables 1, 2 and the L-F
tables, and the convergence orders between successive meshes against the printed ones.  The 1-D
cases use dt = dx/64 (the printed 1-D numbers come from a step far below the stated 0.25 dx; with
it the time error is negligible), the 2-D cases the printed CFL 0.1; the 2-D wave is the diagonal
one the printed norms belong to."""
import math

import numpy as np
import pytest

from paper_2402_10914_gb300 import inputs as I
from tests.test_oracle_scheme import diagonal_wave, golden, norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = (20, 40, 80, 160)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def errors(key, n):
    from paper_2402_10914_gb300.solver import Solver
    flux, scheme = {"gks1d": (I.GKS, I.S2O4), "lf1d": (I.LF, I.SSPRK3),
                    "gks2d": (I.GKS, I.S2O4), "lf2d": (I.LF, I.SSPRK3)}[key]
    if key.endswith("1d"):
        w = I.sine_paper_1d(n, flux=flux, scheme=scheme)
        exact, dt = w.meta["exact"], w.dt_fixed / 16.0
    else:
        w, exact = diagonal_wave(n, flux, scheme)
        dt = 0.0
    with Solver(w.settings) as sol:
        sol.set_ic(w.W0)
        sol.run(t_end=w.t_end, dt=dt, chunk=4096)
        W, _, t, _ = sol.get_state()
    assert t == w.t_end
    return norms(W[0] - exact(t))


def check(key, meshes, tol, order_tol, norms_checked=(0, 1, 2)):
    g = golden()
    errs = [errors(key, n) for n in meshes]
    for n, e in zip(meshes, errs):
        for k in norms_checked:
            assert e[k] == pytest.approx(g[(key, n)][k], rel=tol), (key, n, k, e, g[(key, n)])
    for (n0, e0), (n1, e1) in zip(zip(meshes, errs), zip(meshes[1:], errs[1:])):
        order = math.log2(e0[0] / e1[0])
        printed = math.log2(g[(key, n0)][0] / g[(key, n1)][0])
        assert abs(order - printed) <= order_tol, (key, n1, order, printed)


def test_table_1_gks_1d_all_meshes():
    # measured: 0.7-0.8 % above the printed norms on every mesh, orders equal to 3 decimals
    check("gks1d", MESHES, tol=0.015, order_tol=0.01)


def test_table_2_gks_2d_all_meshes():
    # measured: within 1.2 % of the printed norms on every mesh, orders within 0.003
    check("gks2d", MESHES, tol=0.02, order_tol=0.01)


def test_table_lf1d_meshes_20_to_80():
    # measured: within 1.4 % up to 80 cells; at 160 the SSP-RK3 time error, third order against the
    # fifth-order spatial error, reaches 5 % even at dt = dx/64, so that mesh is left out
    check("lf1d", MESHES[:3], tol=0.02, order_tol=0.03)


def test_table_lf2d_meshes_20_and_40():
    # at the printed CFL 0.1 the SSP-RK3 time error shows from 80 cells on (+4 %, +14 % at 160);
    # the printed 20 x 20 Linf is an outlier of the table (its printed order disagrees with its
    # values), so L1 and L2 are checked
    check("lf2d", MESHES[:2], tol=0.015, order_tol=0.03, norms_checked=(0, 1))


def test_table_lf2d_meshes_80_and_160_lie_between_two_time_steps():
    # The printed L-F 2-D norms at 80 and 160 cells are not reproduced by a smaller time step (the
    # reading that reconciled the 1-D tables): at the printed CFL 0.1 our norms lie above them
    # (SSP-RK3's third-order time error), at CFL 0.025 below them, and a further reduction changes
    # nothing, so the printed numbers come from a step between the two.  Measured: +4.3 % / +14.0 %
    # at CFL 0.1, -6.5 % / -21.4 % at CFL 0.025 (L1, 80 / 160 cells).
    from paper_2402_10914_gb300.solver import Solver
    g = golden()
    for n in (80, 160):
        res = {}
        for cfl in (0.1, 0.025):
            w, exact = diagonal_wave(n, I.LF, I.SSPRK3)
            w.settings = w.settings.with_(cfl=cfl)
            with Solver(w.settings) as sol:
                sol.set_ic(w.W0)
                sol.run(t_end=w.t_end, chunk=8192)
                W, _, t, _ = sol.get_state()
            res[cfl] = norms(W[0] - exact(t))[0] / g[("lf2d", n)][0] - 1.0
        assert 0.0 < res[0.1] < (0.06 if n == 80 else 0.16), (n, res)
        assert (-0.08 if n == 80 else -0.23) < res[0.025] < 0.0, (n, res)
