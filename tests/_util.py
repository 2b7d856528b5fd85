"""Shared helpers for the tests (no method arithmetic)."""
import numpy as np


def rel_err(a, r):
    """Tolerance metric: max_i |a_i - r_i| / (|r_i| + rms(r)).  Plain max relative error is
    ill-posed where a ReLU output is exactly zero, so each element's error is measured against
    its own magnitude plus the RMS of the whole reference."""
    a = np.asarray(a, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if r.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(r * r)))
    if rms == 0.0:
        return float(np.max(np.abs(a - r)))
    return float(np.max(np.abs(a - r) / (np.abs(r) + rms)))


FP32_TOL = 1e-4
BF16_TOL = 2e-2
