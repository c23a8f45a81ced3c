"""Pins of the oracle's reverse-mode adjoint of the stage operator: central finite differences of
the oracle's own stage operator, and the dot-product identity <J v, w> = <v, J^T w>."""
import numpy as np
import pytest

import oracle
from paper_2402_10914_gb300 import inputs as I


def smooth_case(flux, limiter, bc=(I.PERIODIC,) * 4):
    w = I.random_smooth(10, 9, seed=21, amp=0.08, bc=bc, flux=flux, time_limiter=limiter)
    rng = np.random.default_rng(4)
    alpha = rng.uniform(0.3, 1.0, (9, 10))          # fixed; the DF branch depends on alpha only
    return w, alpha


@pytest.mark.parametrize("flux,limiter,bc", [(I.GKS, 1, (I.PERIODIC,) * 4), (I.LF, 0, (I.PERIODIC,) * 4),
                                             (I.GKS, 0, (I.REFLECT, I.REFLECT, I.OUTFLOW, I.OUTFLOW))])
def test_vjp_against_central_differences(flux, limiter, bc):
    w, alpha = smooth_case(flux, limiter, bc)
    s = w.settings
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    rng = np.random.default_rng(9)
    Lb, dLb, dLtb = (rng.normal(size=w.W0.shape) for _ in range(3))
    g = oracle.residual_vjp(s, w.W0, alpha, dt, Lb, dLb, dLtb)

    def J(Wx):
        L, dL, dLt, _, _ = oracle.residual(s, Wx, alpha, dt)
        return (Lb * L).sum() + (dLb * dL).sum() + (dLtb * dLt).sum()
    for _ in range(8):
        k, j, i = rng.integers(0, 4), rng.integers(0, s.ny), rng.integers(0, s.nx)
        h = 1e-6 * max(1.0, abs(w.W0[k, j, i]))
        Wp, Wm = w.W0.copy(), w.W0.copy()
        Wp[k, j, i] += h
        Wm[k, j, i] -= h
        fd = (J(Wp) - J(Wm)) / (2 * h)
        assert g[k, j, i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max()), (k, j, i)


def test_vjp_dot_product_identity():
    # <J v, w> by a directional finite difference equals <v, J^T w>
    w, alpha = smooth_case(I.GKS, 1)
    s = w.settings
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    rng = np.random.default_rng(13)
    v = rng.normal(size=w.W0.shape) * np.abs(w.W0).mean(axis=(1, 2), keepdims=True)
    wb = rng.normal(size=w.W0.shape)
    h = 1e-7
    Lp = oracle.residual(s, w.W0 + h * v, alpha, dt)[0]
    Lm = oracle.residual(s, w.W0 - h * v, alpha, dt)[0]
    lhs = ((Lp - Lm) / (2 * h) * wb).sum()
    rhs = (v * oracle.residual_vjp(s, w.W0, alpha, dt, L_bar=wb)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-6)


@pytest.mark.parametrize("limiter", [0, 1])
def test_step_adjoint_against_central_differences(limiter):
    # three S2O4 steps on smooth data (alpha stays near 1, so the DF branch never acts and holding
    # the alpha sequence fixed is exact); J = <WT_bar, W^n>
    w = I.random_smooth(10, 9, seed=31, amp=0.08, bc=(I.PERIODIC,) * 4, flux=I.GKS, time_limiter=limiter)
    s = w.settings
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    dts = [dt, 0.9 * dt, 1.1 * dt]
    rng = np.random.default_rng(17)
    WTb = rng.normal(size=w.W0.shape)
    WT, g = oracle.run_vjp(s, w.W0, dts, WTb)
    a0 = oracle.alpha0(s, w.W0)
    assert a0.min() > 0.5

    def J(Wx):
        W, a = Wx, a0
        for d in dts:
            rc, W, a, _, _, _ = oracle.run(s, W, a, 1, dt_fixed=d)
            assert rc == 0
        return (WTb * W).sum()
    for _ in range(6):
        k, j, i = rng.integers(0, 4), rng.integers(0, s.ny), rng.integers(0, s.nx)
        # small h: tau_n contains |p_l - p_r|, whose kink at a Gauss point with nearly equal
        # pressures makes a wider difference quotient first-order accurate only
        h = 1e-7 * max(1.0, abs(w.W0[k, j, i]))
        Wp, Wm = w.W0.copy(), w.W0.copy()
        Wp[k, j, i] += h
        Wm[k, j, i] -= h
        fd = (J(Wp) - J(Wm)) / (2 * h)
        assert g[k, j, i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max()), (k, j, i)
