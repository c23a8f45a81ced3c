"""Comparison helpers for GPU-vs-oracle parity tests."""
import numpy as np


def comp_rel_err(a, b, floor_frac=1e-3):
    """max |a-b| / max(|b|, floor_frac * max|b_k|), per component along the first axis."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    worst = 0.0
    for k in range(a.shape[0]):
        scale = np.abs(b[k]).max()
        if scale == 0.0:
            err = np.abs(a[k]).max()
        else:
            err = (np.abs(a[k] - b[k]) / np.maximum(np.abs(b[k]), floor_frac * scale)).max()
        worst = max(worst, float(err))
    return worst


def state_rel_err(a, b, floor_frac=1e-3):
    """Per-cell relative error of a state [4][ny][nx]: plain |a-b|/|b| for density and energy (they
    never cross zero), floored at floor_frac of the component's maximum for the two momenta."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max(axis=(1, 2), keepdims=True)
    den = np.maximum(np.abs(b), floor_frac * scale)
    den[[0, 3]] = np.maximum(np.abs(b[[0, 3]]), 1e-300)
    return np.abs(a - b) / den


def l1_rel(a, b):
    """per-component sum|a-b| / sum|b|, maximum over components."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return max(float(np.abs(a[k] - b[k]).sum() / max(np.abs(b[k]).sum(), 1e-300)) for k in range(a.shape[0]))


def field_err(a, b, floor_frac=1e-3):
    """relative error of a record field array [..., nfield] with a floor per field (last axis)."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), -1, 0)
    b = np.moveaxis(np.asarray(b, dtype=np.float64), -1, 0)
    return comp_rel_err(a, b, floor_frac)


def oracle_envelope(settings, W0, nsteps, t_end=0.0, dt_fixed=0.0, seeds=(101, 202), metric=None, alpha=None):
    """The oracle's own response to rounding-level input noise.

    Runs the oracle from W0 and from W0 * (1 + 1e-15 N(0,1)) (one run per seed) and returns
    (reference run, max per-component relative difference, max relative L1 difference).  Where
    the step map amplifies rounding (the time limiter, strong jumps), no second implementation
    can agree with the oracle more closely than the oracle agrees with itself under this noise.
    alpha: the DF field to start from (default: alpha^0 of W0); metric: a per-cell error function
    for the maximum (default: comp_rel_err)."""
    import oracle
    a0 = oracle.alpha0(settings, W0) if alpha is None else np.asarray(alpha, dtype=np.float64)
    ref = oracle.run(settings, W0, a0, nsteps, dt_fixed=dt_fixed, t_end=t_end)
    worst_max, worst_l1 = 0.0, 0.0
    for sd in seeds:
        rng = np.random.default_rng(sd)
        W2 = W0 * (1.0 + 1e-15 * rng.standard_normal(W0.shape))
        a2 = oracle.alpha0(settings, W2) if alpha is None else a0
        r2 = oracle.run(settings, W2, a2, nsteps, dt_fixed=dt_fixed, t_end=t_end)
        if r2[0] != ref[0] or r2[1].shape != ref[1].shape:
            continue
        worst_max = max(worst_max, comp_rel_err(r2[1], ref[1]) if metric is None else float(metric(r2[1], ref[1]).max()))
        worst_l1 = max(worst_l1, l1_rel(r2[1], ref[1]))
    return ref, worst_max, worst_l1
