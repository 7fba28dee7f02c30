"""Oracle side of the GPU fault sweep, run in spawned worker processes
(imports no torch and touches no GPU)."""
import oracle
from paper_2103_07210_gb300 import inputs


def decisions(o):
    return (o["steps"], tuple(o["detect_steps"]), bool(o["converged"]), o["faults_detected"])


def min_margin(o):
    """Smallest |1 - ||r_t||^2 / ||r_prev||^2| over the fault tests of an oracle
    run whose reference norm the history fixes: step 1 (against ||r^0||^2) and
    every step after an accepted one (against that step's norm).  A step after
    a detected fault tests against the restored backup's norm and is left out,
    as are the exit steps (the exit test comes first) and non-finite norms
    (their test is not close).  Returns inf when no test qualifies."""
    h, ev = o["nrm2_hist"], o["events"]
    best = float("inf")
    for t in range(len(h)):
        if ev[t] == oracle.EVENT_EXIT:
            continue
        if t == 0:
            prev = o["nrm2_0"]
        elif ev[t - 1] == oracle.EVENT_ACCEPT:
            prev = h[t - 1]
        else:
            continue
        if prev > 0 and abs(h[t]) < float("inf"):
            best = min(best, abs(1.0 - h[t] / prev))
    return best


def oracle_trial(args):
    nlon, nlat, k, tol, seed, trial, nff = args
    p = inputs.hill_problem(nlon, nlat)
    f = inputs.sweep_flip(seed, trial, nff, nlon * nlat)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, tol, faults=[f])
    return trial, f, decisions(o), o["faults_injected"], o["x"], min_margin(o)


def fp64_bit_of_fp32_bit(b):
    """The FP64 bit playing the role of FP32 bit b: sign to sign, the exponent's
    low seven bits to the low seven of FP64's, its top bit to FP64's top
    exponent bit, the 23 mantissa bits to the top 23 of FP64's mantissa."""
    if b == 31:
        return 63
    if b == 30:
        return 62
    return b + 29


def oracle_mixed_counterpart(args):
    """FP64 oracle run of a mixed-path trial's flip, bit mapped to FP64."""
    nlon, nlat, k, tol, seed, trial, nsteps = args
    p = inputs.hill_problem(nlon, nlat)
    step, vec, idx, bit = inputs.sweep_flip(seed, trial, nsteps, nlon * nlat, nbits=32)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, tol, faults=[(step, vec, idx, fp64_bit_of_fp32_bit(bit))])
    return trial, o["faults_detected"] > 0, o["converged"]


def oracle_solution(args):
    """FP64 oracle solution of a hill problem: (nlon, nlat, k, tol, rhs, seed,
    hill seed or None for the default hill)."""
    nlon, nlat, k, tol, rhs, seed, hill_seed = args
    hill = inputs.random_hill(hill_seed) if hill_seed is not None else {}
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=seed, **hill)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, tol)
    return o["x"], o["converged"], o["steps"]
