"""Oracle side of the GPU fault sweep, run in spawned worker processes
(imports no torch and touches no GPU)."""
import oracle
from paper_2103_07210_gb300 import inputs


def decisions(o):
    return (o["steps"], tuple(o["detect_steps"]), bool(o["converged"]), o["faults_detected"])


def oracle_trial(args):
    nlon, nlat, k, tol, seed, trial, nff = args
    p = inputs.hill_problem(nlon, nlat)
    f = inputs.sweep_flip(seed, trial, nff, nlon * nlat)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, tol, faults=[f])
    return trial, f, decisions(o), o["faults_injected"], o["x"]
