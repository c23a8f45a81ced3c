"""Pins of the CPU oracle's building blocks against what the paper and mathematics fix.

Each test checks an oracle routine against an independent computation: the paper's printed
interface formulas (Sect. 3.1), exact polynomial reproduction, Gauss-Legendre-free closed forms,
numerical quadrature of Maxwellians, finite differences of the Euler flux, and a brute-force
velocity-space / time quadrature of the paper's interface distribution function (Sect. 2.2).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

GAMMA = 1.4
K = (4 - 2 * GAMMA) / (GAMMA - 1)
RNG = np.random.default_rng(12345)


def cell_avgs_of(f, centres):
    return np.array([integrate.quad(f, c - 0.5, c + 0.5, epsabs=1e-15, epsrel=1e-15)[0] for c in centres])


# ---------------------------------------------------------------- WENO-AO (Sect. 3.1)

def test_sub_polynomials_reproduce_cell_averages():
    Q = RNG.normal(size=5)
    P = oracle.sub_polys(Q)
    stencils = {0: [-2, -1, 0], 1: [-1, 0, 1], 2: [0, 1, 2], 3: [-2, -1, 0, 1, 2]}
    for k, cells in stencils.items():
        p = np.polynomial.Polynomial(P[k])
        for c in cells:
            avg = integrate.quad(p, c - 0.5, c + 0.5)[0]
            assert avg == pytest.approx(Q[c + 2], abs=1e-13)


def test_sub_polynomials_match_printed_interface_forms():
    # Sect. 3.1 prints p^{r3}_0..2 and p^{r5}_3 in x with x = 0 at the interface i+1/2 (xi = 1/2).
    Q = RNG.normal(size=5)
    qm2, qm1, q0, q1, q2 = Q
    P = oracle.sub_polys(Q)
    val = lambda k: np.polynomial.Polynomial(P[k])(0.5)
    der = lambda k: np.polynomial.Polynomial(P[k]).deriv()(0.5)
    der2 = lambda k: np.polynomial.Polynomial(P[k]).deriv(2)(0.5)
    assert val(0) == pytest.approx(qm2 / 3 - 7 * qm1 / 6 + 11 * q0 / 6, abs=1e-13)
    assert der(0) == pytest.approx(qm2 - 3 * qm1 + 2 * q0, abs=1e-13)
    assert der2(0) / 2 == pytest.approx(0.5 * qm2 - qm1 + 0.5 * q0, abs=1e-13)
    assert val(1) == pytest.approx(-qm1 / 6 + 5 * q0 / 6 + q1 / 3, abs=1e-13)
    assert der(1) == pytest.approx(q1 - q0, abs=1e-13)
    assert val(2) == pytest.approx(q0 / 3 + 5 * q1 / 6 - q2 / 6, abs=1e-13)
    assert der(2) == pytest.approx(q1 - q0, abs=1e-13)
    c = [(2 * qm2 - 13 * qm1 + 47 * q0 + 27 * q1 - 3 * q2) / 60,
         (qm1 - 15 * q0 + 15 * q1 - q2) / 12,
         (-qm2 + 6 * qm1 - 8 * q0 + 2 * q1 + q2) / 8,
         (-qm1 + 3 * q0 - 3 * q1 + q2) / 6,
         (qm2 - 4 * qm1 + 6 * q0 - 4 * q1 + q2) / 24]
    p3 = np.polynomial.Polynomial(P[3])
    for n in range(5):
        assert p3.deriv(n)(0.5) / math.factorial(n) == pytest.approx(c[n], abs=1e-12)


def test_smoothness_indicators_closed_forms():
    # Eq. 38 in cell-centred form: quadratics a1^2 + 13/3 a2^2; the quartic's closed form was
    # derived symbolically from the same definition.
    for _ in range(5):
        Q = RNG.normal(size=5)
        P = oracle.sub_polys(Q)
        b = oracle.smoothness(Q)
        for k in range(3):
            a = P[k]
            assert b[k] == pytest.approx(a[1] ** 2 + 13 / 3 * a[2] ** 2, rel=1e-13, abs=1e-14)
        a = P[3]
        b3 = (a[1] ** 2 + a[1] * a[3] / 2 + 13 / 3 * a[2] ** 2 + 21 / 5 * a[2] * a[4]
              + 3129 / 80 * a[3] ** 2 + 87617 / 140 * a[4] ** 2)
        assert b[3] == pytest.approx(b3, rel=1e-13, abs=1e-14)


def test_weno_ao_exact_on_quadratic_data():
    # every sub-stencil polynomial is exact, so any convex weighting returns the quadratic
    coef = RNG.normal(size=3)
    f = np.polynomial.Polynomial(coef)
    Q = cell_avgs_of(f, [-2, -1, 0, 1, 2])
    xi = np.array([-math.sqrt(3) / 6, math.sqrt(3) / 6])
    val, slope, _ = oracle.recon1d(Q, xi)
    assert np.allclose(val, f(xi), atol=1e-12)
    assert np.allclose(slope, f.deriv()(xi), atol=1e-11)


def test_weno_ao_fifth_order_interface_value():
    errs = []
    for h in (0.1, 0.05):
        f = lambda x: np.sin(2.0 + 3.0 * x)
        # Q_s = average of f over [x_s - h/2, x_s + h/2], x_s = s*h; xi = x/h
        Q = np.array([integrate.quad(f, (s - 0.5) * h, (s + 0.5) * h, epsabs=1e-16)[0] / h for s in range(-2, 3)])
        v, _, _ = oracle.recon1d(Q, [0.5])
        errs.append(abs(v[0] - f(0.5 * h)))
    order = math.log2(errs[0] / errs[1])
    assert order > 4.6, order


def test_weno_ao_nonoscillatory_on_step():
    Q = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    v, _, _ = oracle.recon1d(Q, [0.5])
    assert 0.99 < v[0] <= 1.0 + 1e-12      # the smooth left stencil {i-2, i-1, i} dominates


def test_df_quadratic():
    Q = RNG.normal(size=5)
    qm1, q0, q1 = Q[1], Q[2], Q[3]
    # alpha = 1: the DF quadratic is p^{r3}_1
    v, s, _ = oracle.recon1d(Q, [0.5, -0.3], use_df=True, alpha_cell=1.0)
    p1 = np.polynomial.Polynomial(oracle.sub_polys(Q)[1])
    assert np.allclose(v, p1([0.5, -0.3]), atol=1e-13)
    assert np.allclose(s, p1.deriv()([0.5, -0.3]), atol=1e-13)
    # alpha = 0: first order
    v, s, _ = oracle.recon1d(Q, [0.5], use_df=True, alpha_cell=0.0)
    assert v[0] == q0 and s[0] == 0.0
    # Eq. 34's printed form at the interface x = 0 (x0 = -dx/2, x1 = dx^2/3), slope alpha (Q_{i+1}-Q_i)/dx
    a = 0.37
    v, s, _ = oracle.recon1d(Q, [0.5], use_df=True, alpha_cell=a)
    printed = q0 + a * ((q1 - q0) * 0.5 + (0.5 * qm1 - q0 + 0.5 * q1) * (0.0 - 1.0 / 3.0))
    assert v[0] == pytest.approx(printed, abs=1e-13)
    assert s[0] == pytest.approx(a * (q1 - q0), abs=1e-13)
    # zero mean over the cell
    vv, _, _ = oracle.recon1d(Q, np.array([-0.5 + 1e-9, 0.0]), use_df=True, alpha_cell=a)
    gx, gw = np.polynomial.legendre.leggauss(3)
    mean = sum(w * oracle.recon1d(Q, [0.5 * x], use_df=True, alpha_cell=a)[0][0] for x, w in zip(gx, gw)) / 2
    assert mean == pytest.approx(q0, abs=1e-13)


def test_limiter_alpha_smooth_and_rough():
    assert oracle.limiter_alpha(np.array([1e-3, 1e-3, 1e-3, 1e-3])) == 1.0
    b = np.array([1e-8, 5.0, 7.0, 3.0])
    tz = (abs(b[3] - b[0]) + abs(b[3] - b[1]) + abs(b[3] - b[2])) / 3
    a1 = 1 + (tz / (b.min() + 1e-6)) ** 2
    a2 = 1 + (tz / (b.max() + 1e-6)) ** 2
    assert oracle.limiter_alpha(b) == pytest.approx(2 * a2 / (a1 + a2), rel=1e-14)
    assert oracle.limiter_alpha(b) < 1e-6


# ---------------------------------------------------------------- Euler eigensystem, flux Jacobians

def euler_flux_x(W, g=GAMMA):
    rho, m, n, E = W
    u, v = m / rho, n / rho
    p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
    return np.array([m, m * u + p, m * v, u * (E + p)])


def euler_flux_y(W, g=GAMMA):
    rho, m, n, E = W
    u, v = m / rho, n / rho
    p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
    return np.array([n, n * u, n * v + p, v * (E + p)])


def fd_jac(f, W, h=1e-6):
    J = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = h * max(1.0, abs(W[k]))
        J[:, k] = (f(W + e) - f(W - e)) / (2 * e[k])
    return J


def random_state(rng=RNG):
    rho = rng.uniform(0.2, 2.0)
    u, v = rng.uniform(-1.5, 1.5, 2)
    p = rng.uniform(0.1, 2.0)
    return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def test_jacobians_against_finite_differences():
    for _ in range(5):
        W = random_state()
        A, B = oracle.jacobians(W)
        assert np.allclose(A, fd_jac(euler_flux_x, W), rtol=1e-7, atol=1e-7)
        assert np.allclose(B, fd_jac(euler_flux_y, W), rtol=1e-7, atol=1e-7)


def test_characteristic_basis_diagonalises_x_jacobian():
    for _ in range(5):
        W = random_state()
        L, R = oracle.char_basis(W)
        assert np.allclose(L @ R, np.eye(4), atol=1e-12)
        A = fd_jac(euler_flux_x, W)
        rho, u = W[0], W[1] / W[0]
        p = (GAMMA - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / rho)
        c = math.sqrt(GAMMA * p / rho)
        lam = np.diag([u - c, u, u, u + c])
        assert np.allclose(L @ A @ R, lam, atol=1e-6)


# ---------------------------------------------------------------- Maxwellian moments (Sect. 2.2)

def test_moments_against_quadrature():
    for U, lam in [(0.3, 0.7), (-1.2, 2.5), (2.0, 0.3)]:
        dens = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
        full = oracle.moments_u(U, 0.0, lam, 0, K)
        pos = oracle.moments_u(U, 0.0, lam, +1, K)
        neg = oracle.moments_u(U, 0.0, lam, -1, K)
        for n in range(8):
            qp = integrate.quad(lambda u: u ** n * dens(u), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
            qn = integrate.quad(lambda u: u ** n * dens(u), -np.inf, 0, epsabs=1e-14, epsrel=1e-13)[0]
            assert pos[n] == pytest.approx(qp, rel=1e-10, abs=1e-13)
            assert neg[n] == pytest.approx(qn, rel=1e-10, abs=1e-13)
            assert pos[n] + neg[n] == pytest.approx(full[n], rel=1e-12, abs=1e-13)


def psi_matrix_quadrature(W, g=GAMMA):
    """<psi_i psi_j> (normalised) by Gauss-Hermite in u, v and the exact xi moments."""
    rho, u0, v0 = W[0], W[1] / W[0], W[2] / W[0]
    p = (g - 1) * (W[3] - 0.5 * rho * (u0 ** 2 + v0 ** 2))
    lam = rho / (2 * p)
    x, w = np.polynomial.hermite.hermgauss(20)
    us = u0 + x / math.sqrt(lam)
    vs = v0 + x / math.sqrt(lam)
    wu = w / math.sqrt(math.pi)
    xi2, xi4 = K / (2 * lam), K * (K + 2) / (4 * lam ** 2)
    M = np.zeros((4, 4))
    for iu, u in enumerate(us):
        for iv, v in enumerate(vs):
            ww = wu[iu] * wu[iv]
            # psi = (1, u, v, (u^2+v^2+xi^2)/2); average over xi done with its moments
            q = u * u + v * v
            base = np.array([1, u, v, q / 2])
            for i in range(4):
                for j in range(4):
                    if i == 3 and j == 3:
                        val = (q * q + 2 * q * xi2 + xi4) / 4
                    elif i == 3:
                        val = base[j] * (q + xi2) / 2
                    elif j == 3:
                        val = base[i] * (q + xi2) / 2
                    else:
                        val = base[i] * base[j]
                    M[i, j] += ww * val
    return M, lam


def test_slope_solve_against_quadrature_and_closed_form():
    for _ in range(4):
        W = random_state()
        b = RNG.normal(size=4)
        a = oracle.slope_solve(W, b)
        M, lam = psi_matrix_quadrature(W)
        assert np.allclose(M @ a, b, rtol=1e-10, atol=1e-10)
        # closed form (derived symbolically from the same moment system)
        U, V = W[1] / W[0], W[2] / W[0]
        R2, R3 = b[1] - U * b[0], b[2] - V * b[0]
        R4 = 2 * b[3] - (U * U + V * V + (K + 2) / (2 * lam)) * b[0]
        a4 = 4 * lam ** 2 / (K + 2) * (R4 - 2 * U * R2 - 2 * V * R3)
        a3 = 2 * lam * R3 - V * a4
        a2 = 2 * lam * R2 - U * a4
        a1 = b[0] - U * a2 - V * a3 - 0.5 * a4 * (U * U + V * V + (K + 2) / (2 * lam))
        assert np.allclose(a, [a1, a2, a3, a4], rtol=1e-11, atol=1e-11)


def test_time_integrals_against_quadrature():
    # coefficients of the interface distribution (Sect. 2.2) integrated over [0, delta]
    for T, tau, d in [(0.3, 0.0, 0.5), (0.05, 0.05, 0.2), (2.0, 0.7, 0.1)]:
        E = lambda t: math.exp(-t / T)
        coef = [lambda t: 1 - E(t),
                lambda t: (t + tau) * E(t) - tau,
                lambda t: t - tau + tau * E(t),
                lambda t: E(t),
                lambda t: -(tau + t) * E(t),
                lambda t: -tau * E(t)]
        g = oracle.time_integrals(T, tau, d)
        for k in range(6):
            q = integrate.quad(coef[k], 0, d, epsabs=1e-15, epsrel=1e-13)[0]
            assert g[k] == pytest.approx(q, rel=1e-10, abs=1e-14)
    g = oracle.time_integrals(0.0, 0.0, 0.4)
    assert np.allclose(g, [0.4, 0.0, 0.08, 0.0, 0.0, 0.0])


# ---------------------------------------------------------------- GKS flux (Sect. 2.2, 3.4)

def maxwellian_quadrature_nodes(W, n=40, g=GAMMA):
    rho, u0, v0 = W[0], W[1] / W[0], W[2] / W[0]
    p = (g - 1) * (W[3] - 0.5 * rho * (u0 ** 2 + v0 ** 2))
    lam = rho / (2 * p)
    return rho, u0, v0, lam


def brute_force_gks(WL, WLx, WLy, WR, WRx, WRy, dt, C1, C2, tau_reading, g=GAMMA):
    """Eq. 25-27 by direct quadrature: velocity space numerically (Gauss-Legendre on a
    truncated half-line in u, Gauss-Hermite in v, exact xi moments), time integrals of the
    interface distribution's coefficients by scipy.quad."""
    def side(W):
        rho, u0, v0, lam = maxwellian_quadrature_nodes(W)
        return rho, u0, v0, lam

    gh_x, gh_w = np.polynomial.hermite.hermgauss(24)
    gl_x, gl_w = np.polynomial.legendre.leggauss(160)

    def velocity_nodes(state, half):
        rho, u0, v0, lam = state
        s = 1 / math.sqrt(lam)
        if half == 0:
            us = u0 + gh_x * s
            wu = gh_w / math.sqrt(math.pi)
        else:
            lo, hi = (0.0, max(u0, 0) + 12 * s) if half > 0 else (min(u0, 0) - 12 * s, 0.0)
            us = 0.5 * (hi - lo) * gl_x + 0.5 * (hi + lo)
            wu = 0.5 * (hi - lo) * gl_w * math.sqrt(lam / math.pi) * np.exp(-lam * (us - u0) ** 2)
        vs = v0 + gh_x * s
        wv = gh_w / math.sqrt(math.pi)
        return us, wu, vs, wv, K / (2 * lam), K * (K + 2) / (4 * lam ** 2)

    def moment(state, half, poly):
        """rho * int poly(u, v, xi2-moment) * psi g; poly(u, v) returns (c0, c1) with poly = c0 + c1 xi^2."""
        rho = state[0]
        us, wu, vs, wv, x2, x4 = velocity_nodes(state, half)
        out = np.zeros(4)
        for iu, u in enumerate(us):
            for iv, v in enumerate(vs):
                c0, c1 = poly(u, v)
                q = u * u + v * v
                # psi * (c0 + c1 xi^2), averaged over xi
                m0 = c0 + c1 * x2
                m4 = 0.5 * (c0 * (q + x2) + c1 * (q * x2 + x4))
                out += wu[iu] * wv[iv] * np.array([m0, u * m0, v * m0, m4])
        return rho * out

    def a_poly(a, extra=lambda u, v: 1.0):
        return lambda u, v: ((a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v)) * extra(u, v),
                             0.5 * a[3] * extra(u, v))

    def solve(state, b):
        rho, u0, v0, lam = state
        Wloc = np.array([1.0, u0, v0, 0.5 * (u0 ** 2 + v0 ** 2) + (K + 2) / (4 * lam)])
        M, _ = psi_matrix_quadrature(Wloc)
        return np.linalg.solve(M, b)

    sl, sr = side(WL), side(WR)
    alx, aly = solve(sl, WLx / sl[0]), solve(sl, WLy / sl[0])
    arx, ary = solve(sr, WRx / sr[0]), solve(sr, WRy / sr[0])
    one = lambda u, v: (1.0, 0.0)
    Wc = moment(sl, +1, one) + moment(sr, -1, one)
    Wcx = moment(sl, +1, a_poly(alx)) + moment(sr, -1, a_poly(arx))
    Wcy = moment(sl, +1, a_poly(aly)) + moment(sr, -1, a_poly(ary))
    sc = side(Wc)
    acx, acy = solve(sc, Wcx / sc[0]), solve(sc, Wcy / sc[0])
    adv = lambda ax, ay: (lambda u, v: tuple(np.add(a_poly(ax, lambda u, v: u)(u, v), a_poly(ay, lambda u, v: v)(u, v))))
    bt = -moment(sc, 0, adv(acx, acy)) / sc[0]
    Ac = solve(sc, bt)
    Al = solve(sl, -moment(sl, 0, adv(alx, aly)) / sl[0])
    Ar = solve(sr, -moment(sr, 0, adv(arx, ary)) / sr[0])
    pl = (g - 1) * (WL[3] - 0.5 * (WL[1] ** 2 + WL[2] ** 2) / WL[0])
    pr = (g - 1) * (WR[3] - 0.5 * (WR[1] ** 2 + WR[2] ** 2) / WR[0])
    T = C1 * dt + C2 * abs((pl - pr) / (pl + pr)) * dt
    tau = T if tau_reading == 1 else 0.0
    E = lambda t: math.exp(-t / T) if T > 0 else 0.0
    times_u = lambda p: (lambda u, v: tuple(u * c for c in p(u, v)))
    vel = {
        "gc": moment(sc, 0, times_u(one)),
        "ac": moment(sc, 0, times_u(adv(acx, acy))),
        "Ac": moment(sc, 0, times_u(a_poly(Ac))),
        "g": moment(sl, +1, times_u(one)) + moment(sr, -1, times_u(one)),
        "a": moment(sl, +1, times_u(adv(alx, aly))) + moment(sr, -1, times_u(adv(arx, ary))),
        "A": moment(sl, +1, times_u(a_poly(Al))) + moment(sr, -1, times_u(a_poly(Ar))),
    }
    # the second-order interface distribution, term by term (exponent read as e^{-t/tau_n})
    coef = {"gc": lambda t: 1 - E(t), "ac": lambda t: (t + tau) * E(t) - tau,
            "Ac": lambda t: t - tau + tau * E(t), "g": lambda t: E(t),
            "a": lambda t: -(tau + t) * E(t), "A": lambda t: -tau * E(t)}

    def FF(delta):
        tot = np.zeros(4)
        for key in vel:
            tot += integrate.quad(coef[key], 0, delta, epsabs=1e-15, epsrel=1e-13)[0] * vel[key]
        return tot

    F1, F2 = FF(dt), FF(dt / 2)
    return (4 * F2 - F1) / dt, 4 * (F1 - 2 * F2) / dt ** 2


@pytest.mark.parametrize("tau_reading", [0, 1])
def test_gks_point_against_brute_force_quadrature(tau_reading):
    rng = np.random.default_rng(7 + tau_reading)
    for _ in range(2):
        WL, WR = random_state(rng), random_state(rng)
        sl = [rng.normal(scale=0.3, size=4) for _ in range(4)]
        dt = 0.013
        F, dF = oracle.gks_point(WL, sl[0], sl[1], WR, sl[2], sl[3], dt, C1=0.01, C2=5.0, tau_reading=tau_reading)
        Fb, dFb = brute_force_gks(WL, sl[0], sl[1], WR, sl[2], sl[3], dt, 0.01, 5.0, tau_reading)
        assert np.allclose(F, Fb, rtol=1e-8, atol=1e-9), (F, Fb)
        assert np.allclose(dF, dFb, rtol=1e-6, atol=1e-7), (dF, dFb)


def test_gks_uniform_state_gives_euler_flux():
    for _ in range(3):
        W = random_state()
        z = np.zeros(4)
        F, dF = oracle.gks_point(W, z, z, W, z, z, 0.01)
        assert np.allclose(F, euler_flux_x(W), rtol=1e-13, atol=1e-13)
        assert np.allclose(dF, 0.0, atol=1e-10)


def test_gks_equilibrium_limit_gives_cauchy_kovalevskaya_derivative():
    # tau_n = 0 and continuous data: F = Euler flux, dF/dt = A W_t with W_t = -(A W_x + B W_y)
    for _ in range(3):
        W = random_state()
        Wx, Wy = RNG.normal(size=4) * 0.2, RNG.normal(size=4) * 0.2
        F, dF = oracle.gks_point(W, Wx, Wy, W, Wx, Wy, 0.01, C1=0.0, C2=0.0)
        A, B = fd_jac(euler_flux_x, W), fd_jac(euler_flux_y, W)
        Wt = -(A @ Wx + B @ Wy)
        assert np.allclose(F, euler_flux_x(W), rtol=1e-12, atol=1e-12)
        assert np.allclose(dF, A @ Wt, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- L-F flux (Sect. 2.3)

def test_lf_flux_closed_form_and_time_derivative():
    for _ in range(4):
        WL, WR = random_state(), random_state()
        WLx, WLy, WRx, WRy = (RNG.normal(size=4) * 0.3 for _ in range(4))
        F, dF = oracle.lf_point(WL, WLx, WLy, WR, WRx, WRy)

        def speed(W):
            rho, u = W[0], W[1] / W[0]
            p = (GAMMA - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / rho)
            return abs(u) + math.sqrt(GAMMA * p / rho)
        s = max(speed(WL), speed(WR))
        assert np.allclose(F, 0.5 * (euler_flux_x(WL) + euler_flux_x(WR)) - 0.5 * s * (WR - WL), rtol=1e-13, atol=1e-13)
        # time derivative with the wave speed frozen and W_t from the Euler equations on each side
        WtL = -(fd_jac(euler_flux_x, WL) @ WLx + fd_jac(euler_flux_y, WL) @ WLy)
        WtR = -(fd_jac(euler_flux_x, WR) @ WRx + fd_jac(euler_flux_y, WR) @ WRy)
        h = 1e-6
        Fs = lambda t: 0.5 * (euler_flux_x(WL + t * WtL) + euler_flux_x(WR + t * WtR)) - 0.5 * s * ((WR + t * WtR) - (WL + t * WtL))
        assert np.allclose(dF, (Fs(h) - Fs(-h)) / (2 * h), rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- DF factor (Sect. 3.2)

def test_df_alpha_point():
    W = random_state()
    assert oracle.df_alpha_point(W, W) == 1.0
    from paper_2402_10914_gb300.inputs import conserved
    WL = conserved(1.0, 0.5, -0.2, 1.0)
    WR = conserved(0.5, -0.1, 0.3, 0.25)
    cl, cr = math.sqrt(1.4 / 1.0), math.sqrt(1.4 * 0.25 / 0.5)
    D = 0.75 / 1.0 + 0.75 / 0.25 + (0.5 / cl + 0.1 / cr) ** 2 + (-0.2 / cl - 0.3 / cr) ** 2
    assert oracle.df_alpha_point(WL, WR) == pytest.approx(1 / (1 + D * D), rel=1e-14)


def test_df_factor_from_cell_averages_reading():
    # df_states = 1 (an alternative to the paper's reading): both Gauss points of a face take the DF
    # factor of the two cell averages beside it, in the face's local frame; df_states = 0 keeps the
    # reconstructed Gauss-point states
    from paper_2402_10914_gb300 import inputs as I
    w = I.random_rough(9, 7, seed=21)
    s1 = w.settings.with_(df_states=1)
    alpha = np.ones((7, 9))
    for direction in (0, 1):
        faces, _ = oracle.face_records(s1, w.W0, alpha, 1e-3, direction)
        faces0, _ = oracle.face_records(w.settings, w.W0, alpha, 1e-3, direction)
        nt, nf = faces.shape[:2]
        for t in range(nt):
            for f in range(1, nf - 1):                      # faces with interior cells on both sides
                if direction == 0:
                    Wl, Wr = w.W0[:, t, f - 1], w.W0[:, t, f]
                else:                                        # local frame of a y-face: (rho, rhoV, -rhoU, E)
                    Wl = np.array([w.W0[0, f - 1, t], w.W0[2, f - 1, t], -w.W0[1, f - 1, t], w.W0[3, f - 1, t]])
                    Wr = np.array([w.W0[0, f, t], w.W0[2, f, t], -w.W0[1, f, t], w.W0[3, f, t]])
                a = oracle.df_alpha_point(Wl, Wr)
                assert faces[t, f, 9] == a and faces[t, f, 10] == a
                # the fluxes themselves do not depend on where the DF factor comes from
                assert np.array_equal(faces[t, f, :8], faces0[t, f, :8])
        assert not np.array_equal(faces[..., 9], faces0[..., 9])


def test_alpha_from_a_reconstruction_of_the_new_state():
    # alpha_source = 1 (an alternative reading of Algorithm 1's "update DF factor"): alpha^{n+1} is
    # the product of the Gauss-point DF factors (Sect. 3.2) of a reconstruction of W^{n+1} with
    # alpha^n deciding its DF branches -- the stage operator's alpha_next at (W^{n+1}, alpha^n).
    # W^{n+1} and dt do not depend on where alpha^{n+1} comes from.  S2O4 (GKS) and SSP-RK3 (L-F).
    from paper_2402_10914_gb300 import inputs as I
    for w in (I.problem_123(3.0, flux=I.GKS), I.quadrants(24, seed=2), I.problem_123(3.0, flux=I.LF)):
        s0 = w.settings
        s1 = s0.with_(alpha_source=1)
        a0 = oracle.alpha0(s0, w.W0)
        rc0, W_0, a_0, _, dts0, _ = oracle.run(s0, w.W0, a0, 1)
        rc1, W_1, a_1, _, dts1, _ = oracle.run(s1, w.W0, a0, 1)
        assert rc0 == 0 and rc1 == 0
        assert np.array_equal(W_0, W_1) and np.array_equal(dts0, dts1)
        want = oracle.residual(s0, W_1, a0, dts1[0])[3]
        assert np.array_equal(a_1, want)
        assert not np.array_equal(a_1, a_0)                  # the two sources differ on this data
