"""Shared helpers of the GPU parity tests."""
import numpy as np


def rel_err(got, ref, floor=1e-8):
    """max |got - ref| / (|ref| + floor * max|ref|): relative error with a floor
    scaled to the field, for fluxes that span many decades or cross zero."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = np.abs(ref).max()
    if m == 0.0:
        return float(np.abs(got).max())
    return float((np.abs(got - ref) / (np.abs(ref) + floor * m)).max())


def f32_roundtrip(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)
