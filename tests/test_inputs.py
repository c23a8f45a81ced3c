"""The seeded input recipes: cell averages, state ranges, layouts and the flow properties each
workload is defined by (exact cell averages by independent quadrature, a steady vortex in radial
balance, the Mach numbers of the robustness cases).  CPU only; no scheme arithmetic involved."""
import math

import numpy as np
import pytest

from paper_2402_10914_gb300 import inputs as I


def cell_average(f, x0, x1, y0, y1, order=12):
    """Tensor Gauss-Legendre average of f over one cell."""
    g, w = np.polynomial.legendre.leggauss(order)
    xs = 0.5 * (x0 + x1) + 0.5 * (x1 - x0) * g
    ys = 0.5 * (y0 + y1) + 0.5 * (y1 - y0) * g
    X, Y = np.meshgrid(xs, ys)
    return float((np.outer(w, w) * f(X, Y)).sum() / 4.0)


def test_sine_c1_exact_cell_averages():
    w = I.sine_c1(40)
    s = w.settings
    dx = (s.x1 - s.x0) / s.nx
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, j = rng.integers(0, s.nx), rng.integers(0, s.ny)
        ref = cell_average(lambda X, Y: 1.0 + 0.2 * np.sin(np.pi * (X + Y)), i * dx, (i + 1) * dx, j * dx, (j + 1) * dx)
        assert w.W0[0, j, i] == pytest.approx(ref, abs=1e-14)
    # u = v = 1 and p = 1: rho u = rho v = rho, rho E = 1/(gamma-1) + rho
    assert np.array_equal(w.W0[1], w.W0[0]) and np.array_equal(w.W0[2], w.W0[0])
    assert np.allclose(w.W0[3], 1.0 / (s.gamma - 1.0) + w.W0[0], rtol=0, atol=1e-15)
    assert s.bc == (I.PERIODIC,) * 4 and s.flux == I.LF and s.time_limiter == 0 and w.steps == 20


def test_sine_paper_2d_exact_cell_averages():
    w = I.sine_paper_2d(20)
    s = w.settings
    dx = (s.x1 - s.x0) / s.nx
    for i, j in [(0, 0), (3, 17), (11, 5), (19, 19)]:
        ref = cell_average(lambda X, Y: 1.0 + 0.2 * np.sin(np.pi * X) * np.sin(np.pi * Y),
                           s.x0 + i * dx, s.x0 + (i + 1) * dx, s.y0 + j * dx, s.y0 + (j + 1) * dx)
        assert w.W0[0, j, i] == pytest.approx(ref, abs=1e-14)
    # the exact solution at t = 0 is the initial field
    assert np.allclose(w.meta["exact"](0.0), w.W0[0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_quadrants_layout_and_ranges(seed):
    n = 40
    w = I.quadrants(n, seed=seed)
    W = w.W0
    h = n // 2
    # q1 x<.5,y<.5; q2 x>=.5,y<.5; q3 x>=.5,y>=.5; q4 x<.5,y>=.5 (rows are y, columns x)
    blocks = [W[:, :h, :h], W[:, :h, h:], W[:, h:, h:], W[:, h:, :h]]
    for q, (blk, (rho, u, v, p)) in enumerate(zip(blocks, w.meta["states"])):
        assert np.all(blk == blk[:, :1, :1]), q                       # constant in each quadrant
        assert 0.1 <= rho <= 2.0 and -1.5 <= u <= 1.5 and -1.5 <= v <= 1.5 and 0.02 <= p <= 2.0
        r, mu, mv, E = blk[:, 0, 0]
        assert r == rho and mu == pytest.approx(rho * u) and mv == pytest.approx(rho * v)
        assert (E - 0.5 * (mu * mu + mv * mv) / r) * 0.4 == pytest.approx(p)
    again = I.quadrants(n, seed=seed)
    assert np.array_equal(again.W0, W)
    assert not np.array_equal(I.quadrants(n, seed=seed + 10).W0, W)
    s = w.settings
    assert s.bc == (I.OUTFLOW,) * 4 and s.cfl == 0.5 and s.time_limiter == 1 and w.t_end == 0.25


def test_batch_recipe():
    ws = I.batch()
    assert len(ws) == 64
    sides = [w.settings.nx for w in ws]
    assert all(w.settings.nx == w.settings.ny for w in ws) and set(sides) <= set(I.BATCH_SIDES)
    assert len(set(sides)) >= 5                                       # uneven sizes
    fluxes = [w.settings.flux for w in ws]
    assert 16 <= fluxes.count(I.GKS) <= 48                            # both fluxes, roughly half each
    for w in ws:
        s = w.settings
        assert s.bc == (I.OUTFLOW,) * 4 and s.cfl == 0.5 and s.time_scheme == I.S2O4 and w.steps == 200
        assert s.time_limiter == (1 if s.flux == I.GKS else 0)
    assert [w.meta["seed"] for w in ws] == list(range(1000, 1064))
    assert all(np.array_equal(a.W0, b.W0) for a, b in zip(ws[:4], I.batch()[:4]))


def test_vortex_is_a_steady_isentropic_vortex():
    # the recipe's profile: u_theta = eps/(2 pi) exp((1-r^2)/2) r, T = 1 - (gamma-1) eps^2/(8 gamma pi^2)
    # exp(1-r^2), rho = T^(1/(gamma-1)), p = rho T.  Steady in the co-moving frame iff the pressure
    # gradient balances the centripetal term, dp/dr = rho u_theta^2 / r; isentropic: p / rho^gamma = 1.
    g, eps = 1.4, 5.0
    T = lambda r: 1.0 - (g - 1.0) * eps ** 2 / (8.0 * g * math.pi ** 2) * math.exp(1.0 - r * r)
    rho = lambda r: T(r) ** (1.0 / (g - 1.0))
    p = lambda r: rho(r) * T(r)
    ut = lambda r: eps / (2.0 * math.pi) * math.exp(0.5 * (1.0 - r * r)) * r
    for r in (0.3, 0.8, 1.0, 1.7, 2.5):
        h = 1e-5
        dpdr = (p(r + h) - p(r - h)) / (2 * h)
        assert dpdr == pytest.approx(rho(r) * ut(r) ** 2 / r, rel=1e-8)
        assert p(r) / rho(r) ** g == pytest.approx(1.0, rel=1e-13)
    # the generated cell averages (4x4 Gauss points per cell) against a 12x12 rule of the point
    # values: away from the centre, and in the four cells around it (the centre (5,5) is a cell
    # corner at n = 128), where the density is lowest; the background far out
    w = I.vortex(128, noise=0.0)
    W = w.W0
    s = w.settings
    dx = (s.x1 - s.x0) / s.nx

    def rho_xy(X, Y):
        r = np.sqrt((X - 5.0) ** 2 + (Y - 5.0) ** 2)
        return np.vectorize(rho)(r)
    for i, j in [(70, 61), (63, 63), (64, 63), (63, 64), (64, 64)]:
        ref = cell_average(rho_xy, i * dx, (i + 1) * dx, j * dx, (j + 1) * dx)
        assert W[0, j, i] == pytest.approx(ref, rel=1e-9)
    assert W[0].min() == W[0, 63, 63] and W[0].min() == pytest.approx(rho(0.0), rel=5e-3)
    assert W[0, 0, 0] == pytest.approx(1.0, abs=1e-6) and W[1, 0, 0] == pytest.approx(1.0, abs=1e-6)


def test_vortex_noise_is_seeded_density_only():
    a = I.vortex(64, noise=1e-3, seed=7)
    b = I.vortex(64, noise=0.0)
    d = a.W0 - b.W0
    assert np.all(d[1:] == 0.0)
    assert abs(d[0].mean()) < 2e-4 and d[0].std() == pytest.approx(1e-3, rel=0.05)
    assert np.array_equal(I.vortex(64, noise=1e-3, seed=7).W0, a.W0)
    bg = I.vortex_background(64)
    assert np.allclose(bg.W0[1:3], 1.0, atol=0) and np.allclose(bg.W0[0], 1.0, atol=6e-3)


def test_blast_recipe():
    n = 256
    w = I.blast(n)
    s = w.settings
    W = w.W0
    assert np.all(W[0] == 1.0) and np.all(W[1] == 0.0) and np.all(W[2] == 0.0)
    p = W[3] * (s.gamma - 1.0)
    inside = np.isclose(p, 1e4)
    assert np.all(inside | np.isclose(p, 0.01))
    assert inside.sum() == pytest.approx(math.pi * 0.1 ** 2 * n * n, rel=0.02)
    assert s.bc == (I.REFLECT,) * 4 and s.cfl == 0.4 and w.t_end == 0.01


@pytest.mark.parametrize("ma", [2.0, 5.0, 10.0])
def test_robustness_cases_carry_their_mach_numbers(ma):
    w = I.problem_123(ma, n=50)
    W = w.W0
    rho, u = W[0], W[1] / W[0]
    p = (W[3] - 0.5 * rho * u * u) * (w.settings.gamma - 1.0)
    assert np.allclose(np.abs(u) / np.sqrt(w.settings.gamma * p / rho), ma, rtol=1e-12)
    assert np.all(u[:, :25] == -2.0) and np.all(u[:, 25:] == 2.0)
    h = I.hurricane(ma, n=40)
    W = h.W0
    xc, yc, _, _ = I.cell_centres(h.settings)
    X, Y = np.meshgrid(xc, yc)
    u, v = W[1] / W[0], W[2] / W[0]
    speed = np.hypot(u, v)
    p = (W[3] - 0.5 * W[0] * speed ** 2) * (h.settings.gamma - 1.0)
    assert np.allclose(speed / np.sqrt(h.settings.gamma * p / W[0]), ma, rtol=1e-12)
    assert np.allclose(u * X + v * Y, 0.0, atol=1e-12 * speed.max() * 2.0)   # purely rotational
    assert np.allclose(p, 25.0) and np.allclose(W[0], 1.0)


@pytest.mark.parametrize("ma", [0.745, 2.1, 18.1])
def test_planar_rarefaction_reading(ma):
    # the reading of the garbled Sect. 4.3.3 state: every quadrant moves away from the centre with
    # |u| = |v| = 0.6323, all four states on the isentrope p = 1.5 rho^gamma, and the printed
    # reference Mach number sqrt(u^2 + v^2) / sqrt(gamma A rho^(gamma-1)) of the off-diagonal state
    w = I.planar_rarefaction(ma, n=40)
    s = w.settings
    W = w.W0
    xc, yc, _, _ = I.cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    rho, u, v = W[0], W[1] / W[0], W[2] / W[0]
    p = (s.gamma - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
    assert np.allclose(np.abs(u), 0.6323) and np.allclose(np.abs(v), 0.6323)
    assert np.all(np.sign(u) == np.sign(X - 0.5)) and np.all(np.sign(v) == np.sign(Y - 0.5))
    assert np.allclose(p, 1.5 * rho ** s.gamma, rtol=1e-12)
    diag = (X - 0.5) * (Y - 0.5) > 0
    assert np.allclose(rho[diag], 1.0) and np.allclose(p[diag], 1.5)
    off = ~diag
    mach = np.hypot(u, v)[off] / np.sqrt(s.gamma * p[off] / rho[off])
    assert np.allclose(mach, ma, rtol=1e-12)
    assert s.bc == (I.OUTFLOW,) * 4 and w.t_end == 0.15
    if ma == 0.745:                      # the paper's example case, p = 0.4 in the rarefied quadrants
        assert abs(p[off][0] - 0.4) < 2e-3
