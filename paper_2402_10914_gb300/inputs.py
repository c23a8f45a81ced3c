"""Seeded, synthetic initial conditions and run settings for the solver and for the CPU oracle.

This module is the only code the CUDA path and the oracle share.  It holds none of the
scheme's arithmetic: it only builds cell averages of analytic or seeded piecewise-constant
fields (conserved variables W = (rho, rho U, rho V, rho E), SoA [4][ny][nx], x fastest) and the
run settings that go with them.  It imports nothing from the rest of the package.

Workloads (all FP64, gamma = 1.4):
  sine_c1        2-D density wave on periodic [0,2]^2, rho = 1 + 0.2 sin(pi (x+y)), u = v = p = 1,
                 L-F flux, S2O4 without the time limiter, CFL 0.5, 20 steps.
  sine_paper_2d  Sect. 4.1 2-D accuracy case: [-1,1]^2, rho = 1 + 0.2 sin(pi x) sin(pi y),
                 u = v = p = 1, CFL 0.1, t = 2, collision time zero.
  sine_paper_1d  Sect. 4.1 1-D accuracy case on [0,2] (a y-uniform 2-D strip), dt = 0.25 dx, t = 2.
  quadrants      seeded four-quadrant Riemann data on [0,1]^2 split at (0.5, 0.5), states drawn
                 per quadrant (rho ~ U[0.1,2], u, v ~ U[-1.5,1.5], p ~ U[0.02,2]) in the order
                 (x<.5,y<.5), (x>=.5,y<.5), (x>=.5,y>=.5), (x<.5,y>=.5); GKS, outflow, CFL 0.5, t = 0.25.
  batch          64 seeded four-quadrant problems, sides from {64,...,512}, mixed GKS / L-F.
  vortex         isentropic vortex (strength 5 at (5,5)) on periodic [0,10]^2 plus seeded
                 N(0, 1e-3) density noise, GKS, 100 steps.
  blast          pressure ratio 1e6 blast (p = 1e4 inside r < 0.1 of (0.5,0.5), 0.01 outside)
                 on [0,1]^2 with reflecting walls, GKS, CFL 0.4, t = 0.01.
  riemann_cfg3   Sect. 4.2 planar-shock interaction (four constant states split at (0.7,0.7)).
  riemann_cfg6   Sect. 4.2 planar contact interaction on [0,2]^2 (four constant states split at (1,1)).
  problem_123    Sect. 4.3 "123 problem": two receding rarefactions on [0,1] (a y-uniform strip),
                 rho = 1, u = -2 / +2, p0 set by the Mach number u / c, free boundaries, t = 0.14.
  hurricane      Sect. 4.3 hurricane-like flow: rho = 1, p = 25 (entropy A = 25), rotation speed v0
                 set by the Mach number v0 / c0, [-2,2]^2 at dx = 1/100, 50 steps.
  planar_rarefaction  Sect. 4.3.3 interaction of planar rarefaction waves (a reading of the garbled
                 initial state), off-diagonal density set by the Mach number, 400^2, t = 0.15.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC, OUTFLOW, REFLECT = 0, 1, 2
GKS, LF = 0, 1
S2O4, SSPRK3 = 0, 1


@dataclass
class Settings:
    """Mesh, boundary and scheme settings of one problem (mirrors the C configuration struct)."""
    nx: int
    ny: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    gamma: float = 1.4
    cfl: float = 0.5
    bc: tuple = (OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW)   # x-low, x-high, y-low, y-high
    alpha_thres: float = 0.5
    dH: float = 0.85
    dL: float = 0.85
    eps: float = 1e-6
    C1: float = 0.01
    C2: float = 5.0
    flux: int = GKS
    time_limiter: int = 1
    tau_reading: int = 0
    gp_fallback: int = 1
    time_scheme: int = S2O4
    dt_rule: int = 0
    df_states: int = 0                 # DF factor from 0: Gauss-point states, 1: the face's cell averages
    alpha_source: int = 0              # alpha^{n+1} from 0: the last stage, 1: a reconstruction of W^{n+1}

    def with_(self, **kw) -> "Settings":
        return replace(self, **kw)


@dataclass
class Workload:
    name: str
    settings: Settings
    W0: np.ndarray                  # [4][ny][nx] conserved cell averages
    steps: int | None = None        # fixed step count, or None
    t_end: float | None = None      # final time, or None
    dt_fixed: float | None = None   # fixed dt, or None for the CFL rule
    meta: dict = field(default_factory=dict)


def conserved(rho, u, v, p, gamma=1.4):
    """Point values (rho, u, v, p) -> conserved (rho, rho u, rho v, rho E)."""
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def cell_centres(s: Settings):
    dx = (s.x1 - s.x0) / s.nx
    dy = (s.y1 - s.y0) / s.ny
    xc = s.x0 + (np.arange(s.nx) + 0.5) * dx
    yc = s.y0 + (np.arange(s.ny) + 0.5) * dy
    return xc, yc, dx, dy


def _sinc_avg(h):
    """Average of sin(pi x) over a cell of width h, divided by its centre value."""
    a = math.pi * h / 2.0
    return math.sin(a) / a


def sine_c1(n: int = 40) -> Workload:
    s = Settings(nx=n, ny=n, x0=0.0, x1=2.0, y0=0.0, y1=2.0, cfl=0.5,
                 bc=(PERIODIC,) * 4, flux=LF, time_limiter=0)
    xc, yc, dx, dy = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    # exact cell averages of rho = 1 + 0.2 sin(pi (x+y)); rho u = rho v = rho, rho E = p/(g-1) + rho
    rho = 1.0 + 0.2 * _sinc_avg(dx) * _sinc_avg(dy) * np.sin(np.pi * (X + Y))
    W = np.stack([rho, rho, rho, 1.0 / (s.gamma - 1.0) + rho])
    return Workload("sine_c1_%dx%d" % (n, n), s, W, steps=20)


def sine_paper_2d(n: int, flux: int = GKS, scheme: int = S2O4) -> Workload:
    s = Settings(nx=n, ny=n, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, cfl=0.1,
                 bc=(PERIODIC,) * 4, flux=flux, C1=0.0, C2=0.0, time_scheme=scheme)
    xc, yc, dx, dy = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    rho = 1.0 + 0.2 * _sinc_avg(dx) * _sinc_avg(dy) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    W = np.stack([rho, rho, rho, 1.0 / (s.gamma - 1.0) + rho])
    return Workload("sine2d_%d" % n, s, W, t_end=2.0,
                    meta={"exact": lambda t, X=X, Y=Y, dx=dx, dy=dy: 1.0 + 0.2 * _sinc_avg(dx) * _sinc_avg(dy)
                          * np.sin(np.pi * (X - t)) * np.sin(np.pi * (Y - t))})


def sine_paper_1d(n: int, flux: int = GKS, scheme: int = S2O4, ny: int = 4) -> Workload:
    dx = 2.0 / n
    s = Settings(nx=n, ny=ny, x0=0.0, x1=2.0, y0=0.0, y1=ny * dx, cfl=0.5,
                 bc=(PERIODIC,) * 4, flux=flux, C1=0.0, C2=0.0, time_scheme=scheme)
    xc, yc, dx, dy = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    rho = 1.0 + 0.2 * _sinc_avg(dx) * np.sin(np.pi * X)
    W = np.stack([rho, rho, np.zeros_like(rho), 1.0 / (s.gamma - 1.0) + 0.5 * rho])
    return Workload("sine1d_%d" % n, s, W, t_end=2.0, dt_fixed=0.25 * dx,
                    meta={"exact": lambda t, X=X, dx=dx: 1.0 + 0.2 * _sinc_avg(dx) * np.sin(np.pi * (X - t))})


def quadrant_states(rng: np.random.Generator):
    """Four (rho, u, v, p) states drawn in the order q1..q4, each field in the order rho, u, v, p."""
    out = []
    for _ in range(4):
        rho = rng.uniform(0.1, 2.0)
        u = rng.uniform(-1.5, 1.5)
        v = rng.uniform(-1.5, 1.5)
        p = rng.uniform(0.02, 2.0)
        out.append((rho, u, v, p))
    return out


def _four_states(s: Settings, states, xs: float, ys: float):
    xc, yc, _, _ = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    q = np.where(Y < ys, np.where(X < xs, 0, 1), np.where(X >= xs, 2, 3))
    prim = np.array(states, dtype=np.float64)        # [4][rho,u,v,p]
    return conserved(prim[q, 0], prim[q, 1], prim[q, 2], prim[q, 3], s.gamma)


def quadrants(n: int = 400, seed: int = 2, flux: int = GKS, t_end: float = 0.25) -> Workload:
    s = Settings(nx=n, ny=n, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux, time_limiter=1 if flux == GKS else 0)
    states = quadrant_states(np.random.default_rng(seed))
    return Workload("quadrants_%dx%d_seed%d" % (n, n, seed), s, _four_states(s, states, 0.5, 0.5),
                    t_end=t_end, meta={"states": states, "seed": seed})


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batch(count: int = 64, seed_base: int = 1000, steps: int = 200) -> list:
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed_base + k)
        n = BATCH_SIDES[int(rng.uniform() * len(BATCH_SIDES))]
        flux = GKS if rng.uniform() < 0.5 else LF
        states = quadrant_states(rng)
        s = Settings(nx=n, ny=n, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux, time_limiter=1 if flux == GKS else 0)
        out.append(Workload("batch%02d_%d_%s" % (k, n, "gks" if flux == GKS else "lf"), s,
                            _four_states(s, states, 0.5, 0.5), steps=steps, meta={"seed": seed_base + k}))
    return out


def _gl4():
    x, w = np.polynomial.legendre.leggauss(4)
    return 0.5 * x, 0.5 * w


def vortex(n: int = 256, strength: float = 5.0, noise: float = 1e-3, seed: int = 7, steps: int = 100) -> Workload:
    s = Settings(nx=n, ny=n, x0=0.0, x1=10.0, y0=0.0, y1=10.0, cfl=0.5, bc=(PERIODIC,) * 4,
                 flux=GKS, time_limiter=1)
    g = s.gamma
    xc, yc, dx, dy = cell_centres(s)
    gx, gw = _gl4()
    W = np.zeros((4, n, n))
    for a in range(4):
        for b in range(4):
            X, Y = np.meshgrid(xc + gx[a] * dx, yc + gx[b] * dy)
            r2 = (X - 5.0) ** 2 + (Y - 5.0) ** 2
            f = strength / (2 * np.pi) * np.exp(0.5 * (1.0 - r2))
            u = 1.0 - f * (Y - 5.0)
            v = 1.0 + f * (X - 5.0)
            T = 1.0 - (g - 1.0) * strength ** 2 / (8.0 * g * np.pi ** 2) * np.exp(1.0 - r2)
            rho = T ** (1.0 / (g - 1.0))
            W += gw[a] * gw[b] * conserved(rho, u, v, rho * T, g)
    W[0] += np.random.default_rng(seed).normal(0.0, noise, size=(n, n))
    return Workload("vortex_%dx%d" % (n, n), s, W, steps=steps)


def vortex_background(n: int = 256, noise: float = 1e-3, seed: int = 7, steps: int = 100) -> Workload:
    """The vortex case's background flow without the vortex (rho = u = v = p = 1 plus noise)."""
    w = vortex(n, strength=0.0, noise=noise, seed=seed, steps=steps)
    w.name = "vortex_background_%dx%d" % (n, n)
    return w


def blast(n: int = 2048, t_end: float = 0.01) -> Workload:
    s = Settings(nx=n, ny=n, cfl=0.4, bc=(REFLECT,) * 4, flux=GKS, time_limiter=1)
    xc, yc, _, _ = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    inside = (X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.1 ** 2
    p = np.where(inside, 1e4, 0.01)
    W = conserved(np.ones_like(p), np.zeros_like(p), np.zeros_like(p), p, s.gamma)
    return Workload("blast_%dx%d" % (n, n), s, W, t_end=t_end)


def riemann_cfg3(n: int = 500, t_end: float = 0.6, flux: int = GKS) -> Workload:
    """Sect. 4.2 interaction of planar shocks on [0,1]^2; GKS with S2O4 (time limiter on) or L-F
    with SSP-RK3; outflow boundaries."""
    s = Settings(nx=n, ny=n, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux, time_scheme=S2O4 if flux == GKS else SSPRK3)
    states = [(0.138, 1.206, 1.206, 0.129), (0.5323, 0.0, 1.206, 0.3), (1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3)]
    return Workload("riemann3_%dx%d" % (n, n), s, _four_states(s, states, 0.7, 0.7), t_end=t_end)


def riemann_cfg6(n: int = 800, t_end: float = 1.6, flux: int = GKS) -> Workload:
    """Sect. 4.2 interaction of planar contact discontinuities on [0,2]^2 (four constant states split
    at (1,1)); GKS with S2O4 (time limiter on) or L-F with SSP-RK3; outflow boundaries."""
    s = Settings(nx=n, ny=n, x0=0.0, x1=2.0, y0=0.0, y1=2.0, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux,
                 time_scheme=S2O4 if flux == GKS else SSPRK3)
    states = [(1.0, -0.75, 0.5, 1.0), (3.0, -0.75, -0.5, 1.0), (1.0, 0.75, -0.5, 1.0), (2.0, 0.75, 0.5, 1.0)]
    return Workload("riemann6_%dx%d" % (n, n), s, _four_states(s, states, 1.0, 1.0), t_end=t_end)


def problem_123(ma: float, n: int = 100, flux: int = GKS, ny: int = 4) -> Workload:
    """Sect. 4.3, 123 problem: (rho, u, p) = (1, -2, p0) for x < 0.5 and (1, 2, p0) beyond, with p0
    from Ma = |u| / sqrt(gamma p0 / rho); free (outflow) boundaries in x, periodic in y; GKS with
    S2O4 or L-F with SSP-RK3, as the paper pairs them; t = 0.14."""
    dx = 1.0 / n
    s = Settings(nx=n, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=ny * dx, cfl=0.5,
                 bc=(OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), flux=flux, time_scheme=S2O4 if flux == GKS else SSPRK3)
    xc, yc, _, _ = cell_centres(s)
    X, _ = np.meshgrid(xc, yc)
    p0 = 2.0 ** 2 / (s.gamma * ma * ma)
    u = np.where(X < 0.5, -2.0, 2.0)
    W = conserved(np.ones_like(X), u, np.zeros_like(X), np.full_like(X, p0), s.gamma)
    return Workload("p123_ma%g_%d" % (ma, n), s, W, t_end=0.14, meta={"mach": ma, "p0": p0})


def hurricane(ma: float, n: int = 400, flux: int = GKS, steps: int = 50) -> Workload:
    """Sect. 4.3, hurricane-like flow: (rho, u, v, p) = (1, v0 sin(theta), -v0 cos(theta), A rho^gamma)
    with theta the polar angle, A = 25 and v0 from Ma = v0 / c0, c0 = sqrt(gamma A); [-2,2]^2 with
    dx = 1/100 (n = 400) and non-reflecting (outflow) boundaries; 50 steps."""
    s = Settings(nx=n, ny=n, x0=-2.0, x1=2.0, y0=-2.0, y1=2.0, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux,
                 time_scheme=S2O4 if flux == GKS else SSPRK3)
    xc, yc, _, _ = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    A, rho0 = 25.0, 1.0
    p0 = A * rho0 ** s.gamma
    v0 = ma * math.sqrt(s.gamma * p0 / rho0)
    th = np.arctan2(Y, X)
    W = conserved(np.full_like(X, rho0), v0 * np.sin(th), -v0 * np.cos(th), np.full_like(X, p0), s.gamma)
    return Workload("hurricane_ma%g_%d" % (ma, n), s, W, steps=steps, meta={"mach": ma, "v0": v0})


def planar_rarefaction(ma: float, n: int = 400, flux: int = GKS, t_end: float = 0.15) -> Workload:
    """Sect. 4.3.3, interaction of planar rarefaction waves on [0,1]^2 with free (outflow) boundaries,
    dx = 1/400, t = 0.15.  The printed initial state is garbled; read as: (1, -U, -U, 1.5) for
    x < .5, y < .5; (rho, U, -U, A rho^gamma) for x >= .5, y < .5; (1, U, U, 1.5) for x >= .5, y >= .5
    (the printed "1.0.6323" taken as rho = 1.0, u = 0.6323); (rho, -U, U, A rho^gamma) for x < .5,
    y >= .5; U = 0.6323, A = 1.5 (so the rho = 1 quadrants also have p = A rho^gamma).  Every
    quadrant moves away from the centre.  The off-diagonal density rho is the parameter that is
    lowered; it sets the printed reference Mach number sqrt(2) U / sqrt(gamma A rho^(gamma-1)),
    so rho = (2 U^2 / (gamma A Ma^2))^(1/(gamma-1))."""
    s = Settings(nx=n, ny=n, cfl=0.5, bc=(OUTFLOW,) * 4, flux=flux, time_scheme=S2O4 if flux == GKS else SSPRK3)
    U, A = 0.6323, 1.5
    rho = (2.0 * U * U / (s.gamma * A * ma * ma)) ** (1.0 / (s.gamma - 1.0))
    p = A * rho ** s.gamma
    states = [(1.0, -U, -U, 1.5), (rho, U, -U, p), (1.0, U, U, 1.5), (rho, -U, U, p)]
    return Workload("planar_rarefaction_ma%g_%d" % (ma, n), s, _four_states(s, states, 0.5, 0.5), t_end=t_end,
                    meta={"mach": ma, "rho": rho, "p": p})


def random_smooth(nx: int, ny: int, seed: int, amp: float = 0.1, bc=(PERIODIC,) * 4, **kw) -> Workload:
    """A smooth random field (a few low Fourier modes per primitive variable) on [0,1]^2."""
    s = Settings(nx=nx, ny=ny, bc=bc, **kw)
    rng = np.random.default_rng(seed)
    xc, yc, _, _ = cell_centres(s)
    X, Y = np.meshgrid(xc, yc)
    fields = []
    for base in (1.0, 0.3, -0.2, 1.0):
        f = np.full_like(X, base)
        for _ in range(3):
            kx, ky = rng.integers(1, 3, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f = f + amp * rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        fields.append(f)
    return Workload("smooth_%dx%d_seed%d" % (nx, ny, seed), s, conserved(*fields, s.gamma))


def random_rough(nx: int, ny: int, seed: int, bc=(OUTFLOW,) * 4, **kw) -> Workload:
    """Cell-wise random states (rho in [0.2,2], u,v in [-1,1], p in [0.1,2]): discontinuous everywhere."""
    s = Settings(nx=nx, ny=ny, bc=bc, **kw)
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 2.0, (ny, nx))
    u = rng.uniform(-1.0, 1.0, (ny, nx))
    v = rng.uniform(-1.0, 1.0, (ny, nx))
    p = rng.uniform(0.1, 2.0, (ny, nx))
    return Workload("rough_%dx%d_seed%d" % (nx, ny, seed), s, conserved(rho, u, v, p, s.gamma))
