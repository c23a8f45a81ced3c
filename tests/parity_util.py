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
