"""Pins of the oracle's nonlinear WENO-Z weights (Sect. 3.1) and of the time limiter's face weight
(Sect. 2.2) in the regime where their exact values matter.

The smooth accuracy tables fix only the linear limit of the weights, and the step test only their
selectivity; a constant factor inside tau_Z / (beta_k + eps) would pass both.  Here the expected
values are built independently of the oracle's code: the sub-stencil polynomials are typed in the
printed interface form of Sect. 3.1 (x = 0 at the interface x_{i+1/2}, cell i = [-dx, 0], dx = 1),
the smoothness indicators are Eq. 38 integrated symbolically (sympy, exact rationals), and the
weights, tau_Z (Eq. 37) and the AO combination follow the printed formulas in 50-digit arithmetic.
The oracle instead solves the cell-average conditions by Gauss-Jordan elimination and integrates
Eq. 38 by Gauss-Legendre quadrature.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")

X = sp.Symbol("x")
DH = DL = sp.Rational(85, 100)
D3 = DH
D0 = (1 - DH) * (1 - DL) / 2
D1 = (1 - DH) * DL
D2 = D0
EPS = sp.Rational(1, 10 ** 6)


def printed_polys(Q):
    """p^{r3}_0..2 and p^{r5}_3 of Sect. 3.1 in x (dx = 1), from cell averages Q_{i-2..i+2}."""
    qm2, qm1, q0, q1, q2 = [sp.Rational(Fraction(v).limit_denominator(10 ** 12)) if not isinstance(v, sp.Rational)
                            else v for v in Q]
    p0 = (sp.Rational(1, 3) * qm2 - sp.Rational(7, 6) * qm1 + sp.Rational(11, 6) * q0
          + (qm2 - 3 * qm1 + 2 * q0) * X + (sp.Rational(1, 2) * qm2 - qm1 + sp.Rational(1, 2) * q0) * X ** 2)
    p1 = (-sp.Rational(1, 6) * qm1 + sp.Rational(5, 6) * q0 + sp.Rational(1, 3) * q1
          + (q1 - q0) * X + (sp.Rational(1, 2) * qm1 - q0 + sp.Rational(1, 2) * q1) * X ** 2)
    p2 = (sp.Rational(1, 3) * q0 + sp.Rational(5, 6) * q1 - sp.Rational(1, 6) * q2
          + (q1 - q0) * X + (sp.Rational(1, 2) * q0 - q1 + sp.Rational(1, 2) * q2) * X ** 2)
    c0 = sp.Rational(1, 60) * (2 * qm2 - 13 * qm1 + 47 * q0 + 27 * q1 - 3 * q2)
    c1 = sp.Rational(1, 12) * (qm1 - 15 * q0 + 15 * q1 - q2)
    c2 = sp.Rational(1, 8) * (-qm2 + 6 * qm1 - 8 * q0 + 2 * q1 + q2)
    c3 = sp.Rational(1, 6) * (-qm1 + 3 * q0 - 3 * q1 + q2)
    c4 = sp.Rational(1, 24) * (qm2 - 4 * qm1 + 6 * q0 - 4 * q1 + q2)
    p3 = c0 + c1 * X + c2 * X ** 2 + c3 * X ** 3 + c4 * X ** 4
    return [sp.expand(p) for p in (p0, p1, p2, p3)]


def eq38_beta(p):
    """Eq. 38 over cell i = [-1, 0] with dx = 1: sum over derivative orders q of int (d^q p)^2."""
    deg = sp.degree(p, X) if p.has(X) else 0
    return sum(sp.integrate(sp.diff(p, X, q) ** 2, (X, -1, 0)) for q in range(1, deg + 1))


def printed_reconstruction(Q, points):
    """Value and x-derivative of the final AO polynomial (Sect. 3.1) at the given x, plus the four
    smoothness indicators (exact rationals)."""
    P = printed_polys(Q)
    beta = [eq38_beta(p) for p in P]
    with sp.evaluate(True):
        tau = (abs(beta[3] - beta[0]) + abs(beta[3] - beta[1]) + abs(beta[3] - beta[2])) / 3
        d = [D0, D1, D2, D3]
        w = [d[k] * (1 + (tau / (beta[k] + EPS)) ** 2) for k in range(4)]
        s = sum(w)
        wb = [wk / s for wk in w]
        poly = wb[3] * (P[3] / D3 - sum(d[k] / D3 * P[k] for k in range(3))) + sum(wb[k] * P[k] for k in range(3))
    out = []
    for x in points:
        out.append((sp.N(poly.subs(X, x), 50), sp.N(sp.diff(poly, X).subs(X, x), 50)))
    return out, beta


DATA = [
    (0.0, 0.0, 0.0, 1.0, 1.0),              # step between cells i and i+1
    (1.0, 1.0, 0.0, 0.0, 0.0),              # step between cells i-1 and i
    (0.0, 0.0, 1.0, 0.0, 0.0),              # spike in the centre cell
    (0.0, 1.0, 2.0, 2.0, 2.0),              # kink
    (1e-3, 0.0, 2e-3, 1e-3, 0.0),           # amplitude ~1e-3: beta ~ eps, where eps matters
    (3.0, -1.0, 0.5, 4.0, -2.0),            # rough
    (0.0, 0.1, 0.3, 0.2, 0.6),              # moderately rough: no sub-stencil dominates
    (1.0, 1.1, 0.9, 1.4, 1.2),
]
# the data on which the weights are neither linear nor saturated at one sub-stencil
MODERATE = [DATA[2], DATA[4], DATA[5], DATA[6], DATA[7]]


@pytest.mark.parametrize("Q", DATA)
def test_weno_z_weights_in_the_nonlinear_regime(Q):
    # the interface value (x = 0, xi = 1/2) and the Gauss points of the cell (xi = -/+ sqrt(3)/6)
    g = math.sqrt(3.0) / 6.0
    xis = [0.5, -g, g]
    xs = [sp.Rational(0), sp.Float(-g - 0.5, 50), sp.Float(g - 0.5, 50)]
    expect, beta = printed_reconstruction(Q, xs)
    for xi, (v, s) in zip(xis, expect):
        val, slope, b4 = oracle.recon1d(np.array(Q), [xi])
        scale = max(1.0, max(abs(q) for q in Q))
        assert abs(val[0] - float(v)) <= 1e-13 * scale, (Q, xi, val[0], float(v))
        assert abs(slope[0] - float(s)) <= 1e-12 * scale, (Q, xi, slope[0], float(s))
    for k in range(4):
        assert float(beta[k]) == pytest.approx(b4[k], rel=1e-12, abs=1e-300)


def test_weno_z_weight_pin_catches_a_constant_factor_in_the_ratio():
    # the reconstruction with a factor 1.1 inside tau_Z / (beta + eps) differs from the printed one
    # by far more than the tolerance above wherever the weights are neither linear nor saturated on
    # one sub-stencil (at a clean step or kink the smooth stencil takes all the weight either way)
    for Q in MODERATE:
        P = printed_polys(Q)
        beta = [eq38_beta(p) for p in P]
        tau = (abs(beta[3] - beta[0]) + abs(beta[3] - beta[1]) + abs(beta[3] - beta[2])) / 3
        d = [D0, D1, D2, D3]

        def value(fac):
            w = [d[k] * (1 + (sp.nsimplify(fac) * tau / (beta[k] + EPS)) ** 2) for k in range(4)]
            wb = [wk / sum(w) for wk in w]
            poly = wb[3] * (P[3] / D3 - sum(d[k] / D3 * P[k] for k in range(3))) + sum(wb[k] * P[k] for k in range(3))
            return float(sp.N(poly.subs(X, 0), 30))
        assert abs(value(1.1) - value(1)) > 1e-6 * max(abs(q) for q in Q)


def limiter_weight(rho5):
    """alpha^k of the time limiter (Sect. 2.2) for one reconstruction's stencil values: beta_min,
    beta_max over the four indicators, tau_Z of Eq. 37, eps = 1e-6."""
    beta = [eq38_beta(p) for p in printed_polys(rho5)]
    tau = (abs(beta[3] - beta[0]) + abs(beta[3] - beta[1]) + abs(beta[3] - beta[2])) / 3
    a1 = 1 + (tau / (min(beta) + EPS)) ** 2
    a2 = 1 + (tau / (max(beta) + EPS)) ** 2
    return 2 * a2 / (a1 + a2)


def test_time_limiter_weight_on_a_contact_row():
    # A row of cells carrying a pure contact (density varies; u, v, p constant).  In the face
    # line's characteristic basis the entropy variable then equals rho plus a constant, because the
    # entropy eigenvector is (1, u, v, (u^2+v^2)/2) and L = R^{-1}; the other three characteristic
    # variables are constant (their indicators vanish and their limiter weight is 1).  So omega^t of
    # an x-face is min(alpha^L, alpha^R) of the density stencils centred on its left and right cells.
    from paper_2402_10914_gb300 import inputs as I
    gamma = 1.4
    Lb, Rb = oracle.char_basis(np.array([1.3, 1.3 * 0.3, -1.3 * 0.2, 1.0 / 0.4 + 0.5 * 1.3 * 0.13]), gamma)
    u, v = 0.3, -0.2
    assert np.allclose(Rb[:, 1], [1.0, u, v, 0.5 * (u * u + v * v)], atol=1e-15)   # entropy column
    rho = np.array([1.0, 1.0, 1.0, 1.2, 3.0, 3.0, 0.4, 0.5, 0.5, 0.55, 2.0, 2.0, 2.1, 2.05,
                    2.2, 2.35, 2.5, 2.65, 2.8, 2.95, 3.1, 3.25])      # ends on a linear ramp
    nx = rho.size
    s = I.Settings(nx=nx, ny=1, x1=float(nx), y1=1.0, bc=(I.OUTFLOW,) * 4)
    R = rho[None, :]
    W = I.conserved(R, np.full_like(R, u), np.full_like(R, v), np.ones_like(R), gamma)
    faces, _ = oracle.face_records(s, W, np.ones((1, nx)), 1e-3, 0)
    omega = faces.reshape(1, nx + 1, -1)[0, :, 8]
    checked = 0
    for f in range(3, nx - 2):                  # face between cells f-1 and f, stencil f-3 .. f+2
        left = [sp.Rational(Fraction(x).limit_denominator(1000)) for x in rho[f - 3:f + 2]]
        right = [sp.Rational(Fraction(x).limit_denominator(1000)) for x in rho[f - 2:f + 3][::-1]]
        expect = min(limiter_weight(left), limiter_weight(right), sp.Integer(1))
        assert omega[f] == pytest.approx(float(expect), rel=1e-10, abs=1e-15), (f, omega[f], float(expect))
        checked += 1
    assert checked == nx - 5
    # faces at the jumps are strongly limited; inside the linear ramp tau_Z = 0 and omega = 1
    assert omega[3:nx - 2].min() < 1e-6 and omega[nx - 4] == 1.0
