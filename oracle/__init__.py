"""CPU FP64 oracle of the DF + WENO-AO finite-volume scheme -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes + numpy) to ``liboracle.so``, compiled from ``dfgks_oracle.cpp`` with
``g++ -O2 -ffp-contract=off -fopenmp``.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package; the
product path (the CUDA library and its binding) never does.

Arrays follow the product's external layout: conserved W as float64 [4][ny][nx] (x fastest),
alpha as [ny][nx].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfgks_oracle.cpp")
_LIB = os.environ.get("DFGKS_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library in place (plain g++, no fast-math, no FMA contraction)."""
    if os.environ.get("DFGKS_ORACLE_LIB"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc", C.c_int * 4),
                ("alpha_thres", C.c_double), ("dH", C.c_double), ("dL", C.c_double),
                ("eps", C.c_double), ("C1", C.c_double), ("C2", C.c_double),
                ("flux", C.c_int), ("time_limiter", C.c_int), ("tau_reading", C.c_int),
                ("gp_fallback", C.c_int), ("time_scheme", C.c_int), ("dt_rule", C.c_int), ("df_states", C.c_int),
                ("alpha_source", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("fallbacks", C.c_long), ("df_normal", C.c_long), ("df_tangential", C.c_long),
                ("fail_step", C.c_long), ("fail_i", C.c_int), ("fail_j", C.c_int)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            for name in ("oracle_sub_polys", "oracle_smoothness", "oracle_recon1d", "oracle_limiter_alpha",
                         "oracle_char_basis", "oracle_jacobians", "oracle_moments_u", "oracle_slope_solve",
                         "oracle_avg_psi", "oracle_gks_point", "oracle_lf_point", "oracle_df_alpha_point",
                         "oracle_time_integrals", "oracle_fill_ghosts", "oracle_cfl_dt", "oracle_residual",
                         "oracle_face_records", "oracle_alpha0", "oracle_run", "oracle_residual_vjp"):
                getattr(L, name).restype = C.c_int
            L.oracle_moments_u.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, _D]
            L.oracle_gks_point.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int] + [_D] * 8
            L.oracle_lf_point.argtypes = [C.c_double] + [_D] * 8
            L.oracle_df_alpha_point.argtypes = [C.c_double, _D, _D, _D]
            L.oracle_time_integrals.argtypes = [C.c_double, C.c_double, C.c_double, _D]
            L.oracle_recon1d.argtypes = [_D, C.c_int, _D, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_double, _D, _D, _D]
            L.oracle_limiter_alpha.argtypes = [_D, C.c_double, _D]
            L.oracle_char_basis.argtypes = [_D, C.c_double, _D, _D]
            L.oracle_jacobians.argtypes = [_D, C.c_double, _D, _D]
            L.oracle_slope_solve.argtypes = [_D, C.c_double, _D, _D]
            L.oracle_avg_psi.argtypes = [_D, C.c_double, _D, C.c_int, C.c_int, _D]
            L.oracle_residual.argtypes = [C.POINTER(Cfg), _D, _D, C.c_double, _D, _D, _D, _D, C.POINTER(Stats)]
            L.oracle_residual_vjp.argtypes = [C.POINTER(Cfg), _D, _D, C.c_double, _D, _D, _D, _D]
            L.oracle_face_records.argtypes = [C.POINTER(Cfg), _D, _D, C.c_double, C.c_int, _D, _D]
            L.oracle_alpha0.argtypes = [C.POINTER(Cfg), _D, _D]
            L.oracle_run.argtypes = [C.POINTER(Cfg), _D, _D, _D, C.c_int, C.c_double, C.c_double, _D,
                                     C.POINTER(C.c_int), C.POINTER(Stats)]
            L.oracle_fill_ghosts.argtypes = [C.POINTER(Cfg), _D, _D, _D, _D]
            L.oracle_cfl_dt.argtypes = [C.POINTER(Cfg), _D, _D]
            L.oracle_set_threads.argtypes = [C.c_int]
            L.oracle_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


def make_cfg(s) -> Cfg:
    """Build the oracle's configuration from an ``inputs.Settings`` (or any object with its fields)."""
    c = Cfg()
    for f in ("nx", "ny", "x0", "x1", "y0", "y1", "gamma", "cfl", "alpha_thres", "dH", "dL", "eps", "C1", "C2",
              "flux", "time_limiter", "tau_reading", "gp_fallback", "time_scheme", "dt_rule", "df_states",
              "alpha_source"):
        setattr(c, f, getattr(s, f))
    for k in range(4):
        c.bc[k] = int(s.bc[k])
    return c


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return lib().oracle_max_threads()


# ---- unit-level -------------------------------------------------------------------------

def sub_polys(Q):
    out = np.zeros(20)
    lib().oracle_sub_polys(_p(_arr(Q, 5)), _p(out))
    return out.reshape(4, 5)


def smoothness(Q):
    out = np.zeros(4)
    lib().oracle_smoothness(_p(_arr(Q, 5)), _p(out))
    return out


def recon1d(Q, xi, use_df=False, alpha_cell=1.0, dH=0.85, dL=0.85, eps=1e-6):
    xi = _arr(np.atleast_1d(xi))
    val, slope, beta = np.zeros(xi.size), np.zeros(xi.size), np.zeros(4)
    rc = lib().oracle_recon1d(_p(_arr(Q, 5)), xi.size, _p(xi), int(use_df), float(alpha_cell), dH, dL, eps,
                              _p(val), _p(slope), _p(beta))
    assert rc == 0
    return val, slope, beta


def limiter_alpha(beta4, eps=1e-6):
    out = np.zeros(1)
    lib().oracle_limiter_alpha(_p(_arr(beta4, 4)), eps, _p(out))
    return out[0]


def char_basis(W, gamma=1.4):
    L, R = np.zeros(16), np.zeros(16)
    lib().oracle_char_basis(_p(_arr(W, 4)), gamma, _p(L), _p(R))
    return L.reshape(4, 4), R.reshape(4, 4)


def jacobians(W, gamma=1.4):
    A, B = np.zeros(16), np.zeros(16)
    lib().oracle_jacobians(_p(_arr(W, 4)), gamma, _p(A), _p(B))
    return A.reshape(4, 4), B.reshape(4, 4)


def moments_u(U, V, lam, half, K=3.0):
    out = np.zeros(10)
    lib().oracle_moments_u(U, V, lam, half, K, _p(out))
    return out


def slope_solve(W, b, gamma=1.4):
    a = np.zeros(4)
    lib().oracle_slope_solve(_p(_arr(W, 4)), gamma, _p(_arr(b, 4)), _p(a))
    return a


def avg_psi(W, a, i=0, j=0, gamma=1.4):
    out = np.zeros(4)
    lib().oracle_avg_psi(_p(_arr(W, 4)), gamma, _p(_arr(a, 4)), i, j, _p(out))
    return out


def gks_point(WL, WLx, WLy, WR, WRx, WRy, dt, gamma=1.4, C1=0.01, C2=5.0, tau_reading=0):
    F, dF = np.zeros(4), np.zeros(4)
    args = [_p(_arr(v, 4)) for v in (WL, WLx, WLy, WR, WRx, WRy)]
    lib().oracle_gks_point(gamma, C1, C2, dt, tau_reading, *args, _p(F), _p(dF))
    return F, dF


def lf_point(WL, WLx, WLy, WR, WRx, WRy, gamma=1.4):
    F, dF = np.zeros(4), np.zeros(4)
    args = [_p(_arr(v, 4)) for v in (WL, WLx, WLy, WR, WRx, WRy)]
    lib().oracle_lf_point(gamma, *args, _p(F), _p(dF))
    return F, dF


def df_alpha_point(WL, WR, gamma=1.4):
    out = np.zeros(1)
    lib().oracle_df_alpha_point(gamma, _p(_arr(WL, 4)), _p(_arr(WR, 4)), _p(out))
    return out[0]


def time_integrals(T, tau, delta):
    out = np.zeros(6)
    lib().oracle_time_integrals(T, tau, delta, _p(out))
    return out


# ---- scheme-level -----------------------------------------------------------------------

def fill_ghosts(s, W, alpha=None, G=3):
    c = make_cfg(s)
    NG = (s.nx + 2 * G) * (s.ny + 2 * G)
    Wg, ag = np.zeros(4 * NG), np.zeros(NG)
    a = None if alpha is None else _arr(alpha, s.nx * s.ny)
    rc = lib().oracle_fill_ghosts(C.byref(c), _p(_arr(W, 4 * s.nx * s.ny)), _p(a), _p(Wg), _p(ag))
    assert rc == 0
    return Wg.reshape(4, s.ny + 2 * G, s.nx + 2 * G), ag.reshape(s.ny + 2 * G, s.nx + 2 * G)


def cfl_dt(s, W):
    c = make_cfg(s)
    out = np.zeros(1)
    rc = lib().oracle_cfl_dt(C.byref(c), _p(_arr(W, 4 * s.nx * s.ny)), _p(out))
    assert rc == 0
    return out[0]


def residual(s, W, alpha, dt):
    """One stage operator: (L, dL/dt, limited dL/dt, alpha_next, stats)."""
    c = make_cfg(s)
    N = s.nx * s.ny
    L, dL, dLt, an = np.zeros(4 * N), np.zeros(4 * N), np.zeros(4 * N), np.zeros(N)
    st = Stats()
    rc = lib().oracle_residual(C.byref(c), _p(_arr(W, 4 * N)), _p(_arr(alpha, N)), float(dt),
                               _p(L), _p(dL), _p(dLt), _p(an), C.byref(st))
    assert rc == 0, rc
    sh = (4, s.ny, s.nx)
    return L.reshape(sh), dL.reshape(sh), dLt.reshape(sh), an.reshape(s.ny, s.nx), st


def face_records(s, W, alpha, dt, direction):
    """Per-face intermediates (see oracle_face_records); returns (faces[nt][nf][59], lines[nt+4][nf][17])."""
    c = make_cfg(s)
    N = s.nx * s.ny
    nf, nt = (s.nx + 1, s.ny) if direction == 0 else (s.ny + 1, s.nx)
    fo = np.zeros(nf * nt * 59)
    lo = np.zeros(nf * (nt + 4) * 17)
    rc = lib().oracle_face_records(C.byref(c), _p(_arr(W, 4 * N)), _p(_arr(alpha, N)), float(dt), direction,
                                   _p(fo), _p(lo))
    assert rc == 0
    return fo.reshape(nt, nf, 59), lo.reshape(nt + 4, nf, 17)


def alpha0(s, W):
    c = make_cfg(s)
    N = s.nx * s.ny
    out = np.zeros(N)
    rc = lib().oracle_alpha0(C.byref(c), _p(_arr(W, 4 * N)), _p(out))
    assert rc == 0
    return out.reshape(s.ny, s.nx)


def run(s, W, alpha, nsteps, t=0.0, dt_fixed=0.0, t_end=0.0):
    """Advance ``nsteps`` steps (fewer if t_end is reached).  Returns (rc, W, alpha, t, dts, stats)."""
    c = make_cfg(s)
    N = s.nx * s.ny
    Wc = _arr(W, 4 * N).copy()
    ac = _arr(alpha, N).copy()
    tt = np.array([t], dtype=np.float64)
    dts = np.zeros(max(nsteps, 1))
    done = C.c_int(0)
    st = Stats()
    rc = lib().oracle_run(C.byref(c), _p(Wc), _p(ac), _p(tt), int(nsteps), float(dt_fixed or 0.0),
                          float(t_end or 0.0), _p(dts), C.byref(done), C.byref(st))
    return rc, Wc.reshape(4, s.ny, s.nx), ac.reshape(s.ny, s.nx), tt[0], dts[:done.value], st


def residual_vjp(s, W, alpha, dt, L_bar=None, dtL_bar=None, dtLt_bar=None):
    """(dL/dW)^T L_bar + (d dtL/dW)^T dtL_bar + (d dtLt/dW)^T dtLt_bar by reverse-mode
    differentiation of the oracle's stage operator (alpha, dt and branch decisions fixed)."""
    c = make_cfg(s)
    N = s.nx * s.ny
    out = np.zeros(4 * N)
    bars = [None if b is None else _arr(b, 4 * N) for b in (L_bar, dtL_bar, dtLt_bar)]
    rc = lib().oracle_residual_vjp(C.byref(c), _p(_arr(W, 4 * N)), _p(_arr(alpha, N)), float(dt),
                                   _p(bars[0]), _p(bars[1]), _p(bars[2]), _p(out))
    assert rc == 0
    return out.reshape(4, s.ny, s.nx)


def run_vjp(s, W0, dts, WT_bar):
    """The oracle's own reverse sweep through len(dts) S2O4 steps (Eq. 24 with the time limiter):
    each stage's adjoint is residual_vjp, combined by the step's linear structure; alpha^0 from W0,
    the alpha sequence of the forward trajectory held fixed.  Returns (W^n, dJ/dW0)."""
    N = (4, s.ny, s.nx)
    W = np.asarray(W0, dtype=np.float64).reshape(N).copy()
    a = alpha0(s, W)
    hist = []
    for dt in dts:
        L, dL, _, _, _ = residual(s, W, a, dt)
        Ws = W + 0.5 * dt * L + 0.125 * dt * dt * dL
        hist.append((W.copy(), a.copy(), Ws, dt))
        rc, W, a, _, _, _ = run(s, W, a, 1, dt_fixed=dt)
        assert rc == 0
    Wb = np.asarray(WT_bar, dtype=np.float64).reshape(N).copy()
    for Wn, an, Ws, dt in reversed(hist):
        dt2 = dt * dt
        Wsb = residual_vjp(s, Ws, an, dt, dtLt_bar=dt2 / 3.0 * Wb)
        Lb = dt * Wb + 0.5 * dt * Wsb
        dLb = 0.5 * dt2 * Wb + 0.125 * dt2 * Wsb
        dLtb = -dt2 / 3.0 * Wb
        Wb = Wb + Wsb + residual_vjp(s, Wn, an, dt, Lb, dLb, dLtb)
    return W, Wb
