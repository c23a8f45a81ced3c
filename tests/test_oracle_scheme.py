"""Scheme-level pins of the CPU oracle: the paper's printed accuracy tables (Sect. 4.1), exact
invariants of a conservative finite-volume scheme (free stream, conservation, symmetries), the
fourth-order accuracy in time of S2O4 (Eq. 24), boundary maps and positivity on extreme data."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2402_10914_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_accuracy_tables.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        case, n, l1, l2, linf = line.split()
        out[(case, int(n))] = (float(l1), float(l2), float(linf))
    return out


def run_to_end(w, s=None, dt_scale=1.0):
    s = s or w.settings
    a0 = oracle.alpha0(s, w.W0)
    dt = (w.dt_fixed or 0.0) * dt_scale
    rc, W, a, t, dts, st = oracle.run(s, w.W0, a0, 10 ** 7, dt_fixed=dt, t_end=w.t_end)
    assert rc == 0
    return W, a, t, dts, st


def norms(err):
    err = np.abs(err)
    return err.mean(), math.sqrt((err ** 2).mean()), err.max()


def diagonal_wave(n, flux, scheme):
    """Sect. 4.1 2-D accuracy case as the printed tables were produced: rho = 1 + 0.2 sin(pi (x+y)).

    The printed initial condition is the product sin(pi x) sin(pi y), but the printed error norms
    have the ratios of a one-dimensional sinusoid (L2/L1 = 1.111); the diagonal wave reproduces
    Table 2 and Table LF2D to about 1 %, the product form misses them by about 35 %."""
    w = I.sine_paper_2d(n, flux=flux, scheme=scheme)
    xc, yc, dx, dy = I.cell_centres(w.settings)
    X, Y = np.meshgrid(xc, yc)
    S = I._sinc_avg(dx) * I._sinc_avg(dy)
    rho = 1 + 0.2 * S * np.sin(np.pi * (X + Y))
    w.W0 = np.stack([rho, rho, rho, 2.5 + rho])
    return w, (lambda t: 1 + 0.2 * S * np.sin(np.pi * (X + Y - 2 * t)))


# ---------------------------------------------------------------- printed tables

def test_table_lf1d_spatial_error():
    # Table LF1D reproduces with the time error made negligible (dt = dx/64): the reconstruction,
    # characteristic projection and L-F flux are pinned to 1 %.
    g = golden()
    for n in (20,):
        w = I.sine_paper_1d(n, flux=I.LF, scheme=I.SSPRK3)
        W, _, t, _, _ = run_to_end(w, dt_scale=1.0 / 16)
        got = norms(W[0] - w.meta["exact"](t))
        for k in range(3):
            assert got[k] == pytest.approx(g[("lf1d", n)][k], rel=0.01), (k, got, g[("lf1d", n)])


def test_table_1_gks_spatial_error():
    # Table 1 with dt = dx/64: the S2O4 GKS path (collision time zero) within 1.5 %
    g = golden()
    w = I.sine_paper_1d(20, flux=I.GKS)
    W, _, t, _, _ = run_to_end(w, dt_scale=1.0 / 16)
    got = norms(W[0] - w.meta["exact"](t))
    for k in range(3):
        assert got[k] == pytest.approx(g[("gks1d", 20)][k], rel=0.015), (k, got)


@pytest.mark.parametrize("flux,scheme,key,tol", [(I.LF, I.SSPRK3, "lf2d", 0.01), (I.GKS, I.S2O4, "gks2d", 0.02)])
def test_table_2d_accuracy(flux, scheme, key, tol):
    g = golden()
    w, exact = diagonal_wave(20, flux, scheme)
    W, _, t, _, _ = run_to_end(w)
    got = norms(W[0] - exact(t))
    # L1 and L2; the printed 20x20 Linf of Table LF2D is an outlier (its printed order at 40x40
    # is 4.92 while the printed values give 5.56), so Linf is checked for the GKS table only
    kk = (0, 1, 2) if key == "gks2d" else (0, 1)
    for k in kk:
        assert got[k] == pytest.approx(g[(key, 20)][k], rel=tol), (k, got, g[(key, 20)])


def test_convergence_order_lf1d():
    g = golden()
    errs = []
    for n in (20, 40):
        w = I.sine_paper_1d(n, flux=I.LF, scheme=I.SSPRK3)
        W, _, t, _, _ = run_to_end(w, dt_scale=0.25)
        errs.append(norms(W[0] - w.meta["exact"](t))[0])
    order = math.log2(errs[0] / errs[1])
    paper = math.log2(g[("lf1d", 20)][0] / g[("lf1d", 40)][0])
    assert abs(order - paper) < 0.1, (order, paper)
    assert errs[1] == pytest.approx(g[("lf1d", 40)][0], rel=0.02)


# ---------------------------------------------------------------- S2O4 order in time (Eq. 24)

@pytest.mark.parametrize("flux", [I.GKS, I.LF])
def test_s2o4_joint_refinement_order(flux):
    # Eq. 24 at the paper's dt = 0.25 dx (Sect. 4.1): refining mesh and step together keeps the
    # fifth-order spatial rate (Table 1: 4.99 from 20 to 40 cells).  The flux time derivatives are
    # only spatially accurate, so a refinement of dt alone at fixed mesh shows order one; a wrong
    # S2O4 coefficient or time derivative drops the joint rate to two or below.
    errs = []
    for n in (20, 40):
        w = I.sine_paper_1d(n, flux=flux)
        s = w.settings.with_(time_limiter=0)
        W, _, t, _, _ = run_to_end(w, s=s)
        errs.append(norms(W[0] - w.meta["exact"](t))[0])
    order = math.log2(errs[0] / errs[1])
    assert order > 4.6, (order, errs)


def test_time_limiter_off_is_plain_s2o4():
    w = I.random_smooth(12, 10, seed=3, amp=0.05, flux=I.GKS, time_limiter=0)
    s = w.settings
    a = np.ones((s.ny, s.nx))
    dt = 0.3 * oracle.cfl_dt(s, w.W0)
    L1, dL1, _, _, _ = oracle.residual(s, w.W0, a, dt)
    Ws = w.W0 + 0.5 * dt * L1 + 0.125 * dt * dt * dL1
    _, dL2, _, _, _ = oracle.residual(s, Ws, a, dt)
    expect = w.W0 + dt * L1 + dt * dt / 6 * (dL1 + 2 * dL2)
    rc, W, _, _, _, _ = oracle.run(s, w.W0, a, 1, dt_fixed=dt)
    assert rc == 0
    assert np.allclose(W, expect, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("flux", [I.GKS, I.LF])
@pytest.mark.parametrize("bc", [(I.PERIODIC,) * 4, (I.OUTFLOW,) * 4])
def test_free_stream_is_preserved_bitwise(flux, bc):
    s = I.Settings(nx=9, ny=7, bc=bc, flux=flux)
    W0 = np.broadcast_to(I.conserved(0.7, 0.3, -0.4, 1.3)[:, None, None], (4, 7, 9)).copy()
    rc, W, a, _, _, _ = oracle.run(s, W0, np.ones((7, 9)), 3)
    assert rc == 0
    assert np.array_equal(W, W0)


def test_reflecting_box_at_rest_is_preserved():
    s = I.Settings(nx=8, ny=8, bc=(I.REFLECT,) * 4, flux=I.GKS)
    W0 = np.broadcast_to(I.conserved(1.1, 0.0, 0.0, 0.9)[:, None, None], (4, 8, 8)).copy()
    rc, W, _, _, _, _ = oracle.run(s, W0, np.ones((8, 8)), 2)
    assert rc == 0 and np.array_equal(W, W0)


@pytest.mark.parametrize("flux", [I.GKS, I.LF])
def test_periodic_conservation(flux):
    w = I.random_rough(16, 12, seed=5, bc=(I.PERIODIC,) * 4, flux=flux)
    a0 = oracle.alpha0(w.settings, w.W0)
    rc, W, _, _, _, st = oracle.run(w.settings, w.W0, a0, 3)
    assert rc == 0
    tot0, tot = w.W0.sum(axis=(1, 2)), W.sum(axis=(1, 2))
    assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(w.W0).sum(axis=(1, 2)))


def transpose_field(W):
    return np.stack([W[0].T, W[2].T, W[1].T, W[3].T])


@pytest.mark.parametrize("flux", [I.GKS, I.LF])
def test_xy_transpose_symmetry(flux):
    w = I.random_rough(14, 11, seed=9, flux=flux)
    s = w.settings
    sT = s.with_(nx=s.ny, ny=s.nx, x0=s.y0, x1=s.y1, y0=s.x0, y1=s.x1, bc=(s.bc[2], s.bc[3], s.bc[0], s.bc[1]))
    a0 = oracle.alpha0(s, w.W0)
    a0T = oracle.alpha0(sT, transpose_field(w.W0))
    assert np.allclose(a0T, a0.T, rtol=1e-13, atol=1e-15)
    dt = 0.5 * oracle.cfl_dt(s, w.W0)
    rc, W, a, _, _, _ = oracle.run(s, w.W0, a0, 2, dt_fixed=dt)
    rcT, WT, aT, _, _, _ = oracle.run(sT, transpose_field(w.W0), a0T, 2, dt_fixed=dt)
    assert rc == 0 and rcT == 0
    assert np.allclose(WT, transpose_field(W), rtol=1e-12, atol=1e-13)
    assert np.allclose(aT, a.T, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("flux", [I.GKS, I.LF])
def test_x_mirror_symmetry(flux):
    w = I.random_rough(13, 9, seed=21, flux=flux)
    s = w.settings
    mirror = lambda W: np.stack([W[0][:, ::-1], -W[1][:, ::-1], W[2][:, ::-1], W[3][:, ::-1]])
    dt = 0.5 * oracle.cfl_dt(s, w.W0)
    a0 = oracle.alpha0(s, w.W0)
    rc, W, _, _, _, _ = oracle.run(s, w.W0, a0, 2, dt_fixed=dt)
    rcM, WM, _, _, _, _ = oracle.run(s, mirror(w.W0), oracle.alpha0(s, mirror(w.W0)), 2, dt_fixed=dt)
    assert rc == 0 and rcM == 0
    assert np.allclose(WM, mirror(W), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- boundaries, DF, positivity

@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (0, 0, 2, 1), (1, 2, 0, 0)])
def test_ghost_maps(bc):
    G = 3
    s = I.Settings(nx=5, ny=4, bc=bc)
    rng = np.random.default_rng(1)
    W = rng.uniform(0.5, 1.5, (4, 4, 5))
    alpha = rng.uniform(0, 1, (4, 5))
    Wg, ag = oracle.fill_ghosts(s, W, alpha)

    def src(k, n, lo, hi):
        if 0 <= k < n:
            return k, 1
        b = lo if k < 0 else hi
        if b == 0:
            return k % n, 1
        if b == 1:
            return (0 if k < 0 else n - 1), 1
        return (-1 - k if k < 0 else 2 * n - 1 - k), -1
    for jj in range(-G, 4 + G):
        for ii in range(-G, 5 + G):
            i, sx = src(ii, 5, bc[0], bc[1])
            j, sy = src(jj, 4, bc[2], bc[3])
            expect = W[:, j, i] * np.array([1, sx, sy, 1])
            assert np.array_equal(Wg[:, jj + G, ii + G], expect), (ii, jj)
            assert ag[jj + G, ii + G] == alpha[j, i]


def test_alpha_is_one_on_uniform_data_and_in_range_on_rough_data():
    s = I.Settings(nx=6, ny=6)
    W0 = np.broadcast_to(I.conserved(1.0, 0.2, 0.1, 1.0)[:, None, None], (4, 6, 6)).copy()
    assert np.all(oracle.alpha0(s, W0) == 1.0)
    w = I.random_rough(10, 10, seed=4)
    a = oracle.alpha0(w.settings, w.W0)
    assert np.all((a > 0) & (a <= 1))
    assert (a < 0.5).mean() > 0.5


def test_df_branch_fires_on_rough_data():
    w = I.random_rough(12, 12, seed=8)
    s = w.settings
    a = np.full((12, 12), 0.2)
    _, _, _, _, st = oracle.residual(s, w.W0, a, 1e-3)
    assert st.df_normal > 0 and st.df_tangential > 0
    _, _, _, _, st1 = oracle.residual(s, w.W0, np.ones((12, 12)), 1e-3)
    assert st1.df_normal == 0 and st1.df_tangential == 0


def test_blast_positivity_small():
    w = I.blast(n=48, t_end=0.002)
    a0 = oracle.alpha0(w.settings, w.W0)
    rc, W, a, t, dts, st = oracle.run(w.settings, w.W0, a0, 40, t_end=w.t_end)
    assert rc == 0
    g = w.settings.gamma
    p = (g - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
    assert W[0].min() > 0 and p.min() > 0
    # reflecting walls conserve mass exactly and the blast is symmetric under x <-> y
    assert abs(W[0].sum() - w.W0[0].sum()) <= 1e-13 * w.W0[0].sum()
    assert np.allclose(W[0], W[0].T, rtol=1e-12)


@pytest.mark.parametrize("rule", [0, 1])
def test_cfl_step_closed_forms(rule):
    # a uniform moving state on a non-square mesh: dt = CFL * min(dx/(|U|+c), dy/(|V|+c)) (rule 0)
    # or CFL / ((|U|+c)/dx + (|V|+c)/dy) (rule 1), with c = sqrt(gamma p / rho)
    s = I.Settings(nx=12, ny=7, x1=2.0, y1=0.5, cfl=0.45, dt_rule=rule)
    rho, u, v, p = 1.3, -0.7, 0.4, 2.1
    W = np.broadcast_to(I.conserved(rho, u, v, p, s.gamma)[:, None, None], (4, s.ny, s.nx)).copy()
    c = np.sqrt(s.gamma * p / rho)
    dx, dy = 2.0 / 12, 0.5 / 7
    want = min(dx / (abs(u) + c), dy / (abs(v) + c)) if rule == 0 else 1.0 / ((abs(u) + c) / dx + (abs(v) + c) / dy)
    assert oracle.cfl_dt(s, W) == pytest.approx(s.cfl * want, rel=1e-14)


def test_robustness_inputs_have_their_mach_numbers():
    # the 123 problem and the hurricane-like flow are parametrised by a Mach number (Sect. 4.3)
    g = 1.4
    for ma in (2.0, 31.5):
        w = I.problem_123(ma)
        rho, u = w.W0[0], w.W0[1] / w.W0[0]
        p = (g - 1) * (w.W0[3] - 0.5 * rho * u * u)
        assert np.allclose(np.abs(u) / np.sqrt(g * p / rho), ma, rtol=1e-12)
        assert np.all(u[:, : w.settings.nx // 2] == -2.0) and np.all(u[:, w.settings.nx // 2:] == 2.0)
        h = I.hurricane(ma, n=40)
        rho, u, v = h.W0[0], h.W0[1] / h.W0[0], h.W0[2] / h.W0[0]
        p = (g - 1) * (h.W0[3] - 0.5 * rho * (u * u + v * v))
        assert np.allclose(np.hypot(u, v) / np.sqrt(g * p / rho), ma, rtol=1e-12)
        xc, yc, _, _ = I.cell_centres(h.settings)
        X, Y = np.meshgrid(xc, yc)
        assert np.allclose(u * X + v * Y, 0.0, atol=1e-9 * ma)        # purely azimuthal
        assert np.all(u * Y - v * X > 0)                              # rotating clockwise: (u, v) = v0 (sin, -cos)


@pytest.mark.parametrize("nx,ny,bc", [(2, 6, (I.REFLECT, I.REFLECT, I.OUTFLOW, I.OUTFLOW)),
                                      (6, 2, (I.OUTFLOW, I.OUTFLOW, I.REFLECT, I.REFLECT)),
                                      (2, 6, (I.PERIODIC,) * 4)])
def test_oracle_refuses_walls_and_wraps_on_fewer_than_three_cells(nx, ny, bc):
    # a reflecting wall mirrors ghost k onto interior cell k (k < 3), a periodic wrap copies the
    # opposite 3 cells: with fewer interior cells the map would read other ghost cells
    w = I.random_smooth(nx, ny, 1, bc=bc, flux=I.GKS)
    with pytest.raises(AssertionError):
        oracle.alpha0(w.settings, w.W0)
    ok = I.random_smooth(3 if nx == 2 else nx, 3 if ny == 2 else ny, 1, bc=bc, flux=I.GKS)
    assert np.all(np.isfinite(oracle.alpha0(ok.settings, ok.W0)))
