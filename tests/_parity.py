"""Shared helpers of the GPU parity tests.

The flux of a DFEM sweep crosses zero (the method allows negative nodal values)
and spans many decades, so a pointwise relative error is ill-posed at nodes
near zero.  The parity bar is the per-group max-norm relative error
||phi_g - ref_g||_inf / ||ref_g||_inf; pointwise relative errors are reported
only where |ref| is at least a fraction of the group maximum."""
import numpy as np


def norm_err(got, ref):
    """max over groups of ||got_g - ref_g||_inf / ||ref_g||_inf (arrays [G, ...] or [...])."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim < 3:
        got, ref = got[None], ref[None]
    worst = 0.0
    for g in range(ref.shape[0]):
        m = np.abs(ref[g]).max()
        d = np.abs(got[g] - ref[g]).max()
        worst = max(worst, d / m if m > 0 else d)
    return float(worst)


def point_err(got, ref, floor=1e-2):
    """max |got - ref| / |ref| over nodes with |ref| >= floor * group max."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim < 3:
        got, ref = got[None], ref[None]
    worst = 0.0
    for g in range(ref.shape[0]):
        m = np.abs(ref[g]).max()
        sel = np.abs(ref[g]) >= floor * m
        if sel.any():
            worst = max(worst, float((np.abs(got[g] - ref[g])[sel] / np.abs(ref[g])[sel]).max()))
    return worst


def rel_err(got, ref):
    """The parity measure used by the GPU tests (see the module docstring)."""
    return norm_err(got, ref)


def f32_roundtrip(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)
