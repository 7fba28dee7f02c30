"""Helpers shared by the GPU parity tests (comparison rules only)."""
import numpy as np


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """Relative 2-norm error of a against reference b over the finite
    entries; non-finite entries must coincide exactly (same NaN / same
    signed Inf positions), otherwise +inf is returned."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    if not np.array_equal(np.isnan(a), np.isnan(b)):
        return float("inf")
    ia, ib = np.isinf(a), np.isinf(b)
    if not np.array_equal(ia, ib) or not np.array_equal(np.sign(a[ia]), np.sign(b[ib])):
        return float("inf")
    f = np.isfinite(b)
    scale = np.abs(b[f]).max() if f.any() else 0.0
    if scale == 0.0:
        return float(np.abs(a[f]).max()) if f.any() else 0.0
    nb = np.linalg.norm(b[f] / scale)
    d = np.linalg.norm(a[f] / scale - b[f] / scale)
    return float(d / nb)


def decisions(info: dict) -> tuple:
    """What must match exactly between the GPU FP64 path and the oracle."""
    return (info["steps"], tuple(info["detect_steps"]), bool(info["converged"]), info["faults_detected"])
