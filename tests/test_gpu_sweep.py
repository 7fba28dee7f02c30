"""Fault sweep at 512 x 256 (FP64, k = 4, hill coefficients, flow RHS): 1000
seeded single-bit flips, uniform over step (1..fault-free step count),
vector {x, r, p, Ap}, index and bit 0-63.  The GPU path must take exactly the
oracle's decisions (detected or not, detection steps, step count,
convergence) and match its solution to 1e-10 (an undetected flip of an x or
p entry stays confined to that entry of the solution, whose value is its
pre-flip rounding scaled by the flip: that entry is left out).  The smallest fault-test margin
|1 - ||r_t||^2 / ||r_prev||^2| over the sweep is printed: the distance from
the closest decision to a tie, against which the double-double reductions'
error (about N 2^-106) is judged."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests import sweep_worker
from tests.gpu_util import decisions, rel_err_fault_trial

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NLON, NLAT, K, TOL, SEED, TRIALS = 512, 256, 4, 1e-10, 0, 1000


def test_sweep_1000_flips_identical_decisions():
    p = inputs.hill_problem(NLON, NLAT)
    ff = oracle.ftgcr(p.D, p.R, p.mu, K, TOL)
    nff = ff["steps"]
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        refs = pool.map(sweep_worker.oracle_trial, [(NLON, NLAT, K, TOL, SEED, t, nff) for t in range(TRIALS)],
                        chunksize=8)
    mism, worst, detected, worst_case = [], 0.0, 0, None
    margin = min(r[5] for r in refs)
    with ftgcr.Solver(p.D, p.mu, k=K, tol=TOL) as s:
        R = torch.from_numpy(p.R).cuda()
        for trial, f, dref, inj, xref, _ in refs:
            x = torch.zeros_like(R)
            s.solve(R, x, faults=[f])
            info = s.stats()
            if decisions(info) != dref or info["faults_injected"] != inj:
                mism.append((trial, f, decisions(info), dref))
                continue
            detected += info["faults_detected"] > 0
            e = rel_err_fault_trial(x.cpu().numpy(), xref, f, info["faults_detected"] > 0)
            if e > worst:
                worst, worst_case = e, (trial, f, float(np.abs(xref[np.isfinite(xref)]).max()))
    print(f"{TRIALS} flips: {detected} detected, identical decisions; smallest fault-test margin {margin:.3e}; "
          f"worst solution error {worst:.2e}")
    assert not mism, mism[:5]
    assert worst <= 1e-10, (worst, worst_case)
    assert detected > 0
    # the closest decision is many FP64 ulps from a tie, so identical
    # decisions do not rest on the two sides rounding their dots alike
    assert margin > 1e-14, margin
