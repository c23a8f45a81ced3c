"""Hand-written GPU adjoint against the oracle's reverse-mode adjoint, finite differences and the
dot-product identity (alpha, dt and branch decisions fixed by the forward pass)."""
import numpy as np
import pytest

import oracle
from paper_2402_10914_gb300 import inputs as I
from tests.parity_util import comp_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


CASES = {
    "gks_limiter_rough": lambda: (I.random_rough(14, 11, seed=41, flux=I.GKS, time_limiter=1), "random"),
    "gks_smooth_reflect": lambda: (I.random_smooth(14, 11, seed=42, bc=(I.REFLECT, I.REFLECT, I.OUTFLOW, I.OUTFLOW),
                                                   flux=I.GKS, time_limiter=1), "ones"),
    "gks_tau_n": lambda: (I.random_smooth(14, 11, seed=43, flux=I.GKS, time_limiter=0, tau_reading=1), "ones"),
    "lf_periodic_rough": lambda: (I.random_rough(14, 11, seed=44, bc=(I.PERIODIC,) * 4, flux=I.LF, time_limiter=0),
                                  "random"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_stage_vjp_matches_oracle(name):
    from paper_2402_10914_gb300.solver import Solver, adjoint_residual
    w, akind = CASES[name]()
    s = w.settings
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0.0, 1.0, (s.ny, s.nx)) if akind == "random" else np.ones((s.ny, s.nx))
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    Lb, dLb, dLtb = (rng.normal(size=w.W0.shape) for _ in range(3))
    ref = oracle.residual_vjp(s, w.W0, alpha, dt, Lb, dLb, dLtb)
    with Solver(s) as sol:
        got = host(adjoint_residual(sol, w.W0, alpha, dt, Lb, dLb, dLtb))
    assert comp_rel_err(got, ref) <= 1e-9, comp_rel_err(got, ref)


def test_stage_vjp_dot_product_identity():
    # <J v, w> by a directional difference of the GPU stage operator = <v, J^T w> by the GPU adjoint
    from paper_2402_10914_gb300.solver import Solver, adjoint_residual
    w = I.random_smooth(24, 20, seed=45, flux=I.GKS, time_limiter=1)
    s = w.settings
    alpha = np.ones((s.ny, s.nx))
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    rng = np.random.default_rng(6)
    v = rng.normal(size=w.W0.shape) * np.abs(w.W0).mean(axis=(1, 2), keepdims=True)
    wb = rng.normal(size=w.W0.shape)
    h = 1e-7
    with Solver(s) as sol:
        Lp = host(sol.residual(dev(w.W0 + h * v), dev(alpha), dt)[0])
        Lm = host(sol.residual(dev(w.W0 - h * v), dev(alpha), dt)[0])
        g = host(adjoint_residual(sol, w.W0, alpha, dt, L_bar=wb))
    lhs = ((Lp - Lm) / (2 * h) * wb).sum()
    rhs = (v * g).sum()
    assert lhs == pytest.approx(rhs, rel=1e-6)


@pytest.mark.parametrize("limiter", [0, 1])
def test_step_adjoint_matches_oracle(limiter):
    # 6 steps with a checkpoint every 4 (two recomputed segments) against the oracle's reverse sweep
    from paper_2402_10914_gb300.solver import Solver, adjoint_steps
    w = I.random_smooth(16, 12, seed=46, flux=I.GKS, time_limiter=limiter)
    s = w.settings
    dt = 0.4 * oracle.cfl_dt(s, w.W0)
    dts = [dt * f for f in (1.0, 0.9, 1.1, 1.0, 0.95, 1.05)]
    WTb = np.random.default_rng(7).normal(size=w.W0.shape)
    WT, ref = oracle.run_vjp(s, w.W0, dts, WTb)
    with Solver(s) as sol:
        got = host(adjoint_steps(sol, w.W0, dts, WTb, ckpt_every=4))
        W, _, t, step = sol.get_state()
    assert comp_rel_err(got, ref) <= 1e-9, comp_rel_err(got, ref)
    assert step == 6 and comp_rel_err(W, WT) <= 1e-12


def run_fixed(sol, W0, dts):
    sol.set_ic(W0)
    for d in dts:
        sol.step(1, dt=float(d))
    return sol.get_state()[0]


def test_autograd_function_and_finite_differences():
    from paper_2402_10914_gb300.solver import GKSRun, Solver
    w = I.vortex(32, steps=8)
    s = w.settings
    with Solver(s) as sol:
        W0 = dev(w.W0).requires_grad_(True)
        WT = GKSRun.apply(W0, sol, 8, 3)
        J = (WT[0] ** 2).sum()
        J.backward()
        g = host(W0.grad)
        sol.set_ic(w.W0)
        _, dts = sol.step(8, record_dts=True)
        rng = np.random.default_rng(8)
        for _ in range(6):
            k, j, i = rng.integers(0, 4), rng.integers(0, s.ny), rng.integers(0, s.nx)
            h = 1e-7 * max(1.0, abs(w.W0[k, j, i]))
            Wp, Wm = w.W0.copy(), w.W0.copy()
            Wp[k, j, i] += h
            Wm[k, j, i] -= h
            fd = ((run_fixed(sol, Wp, dts)[0] ** 2).sum() - (run_fixed(sol, Wm, dts)[0] ** 2).sum()) / (2 * h)
            assert g[k, j, i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max()), (k, j, i)
