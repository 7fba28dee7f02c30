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



def rel_err_fault_trial(a: np.ndarray, b: np.ndarray, fault, detected: bool) -> float:
    """Solution error of a single-flip trial.  x and p enter neither beta,
    alpha nor the residual recurrences (Algorithm 1), so a flip of an x or p
    entry is never detected and stays confined to that entry of the solution
    (Section 3: such faults are passive); its value there is the entry's
    pre-flip rounding scaled by the flip (by up to 2^1024 for an exponent
    bit), so two implementations that round differently agree there only to
    that scaled rounding.  That entry is left out; every other entry must
    match.  fault = (step, vec, index, bit)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    step, vec, idx, bit = fault
    if not detected and vec in (0, 2):  # x, p
        keep = np.ones(a.size, dtype=bool)
        keep[idx] = False
        return rel_err(a[keep], b[keep])
    return rel_err(a, b)
