"""Mixed path under single-bit faults at the benchmark size (1024 x 512 hill
problem, k = 4 and 8): 100 and 50 seeded flips of FP32 inner vectors (x, r,
p, Ap; bit 0-31) in the first refinement sweep's inner steps.  Every solve
must converge to the fault-free FP64 oracle solution within 1e-10 (tol
1e-13).  The exact-decision requirement binds the FP64 path only; here the
test reports how often the mixed path's detection agrees with the oracle's
for the same flip at the corresponding FP64 bit, and asserts only that
agreement is the usual case."""
import multiprocessing as mp
import os

import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests import sweep_worker
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NLON, NLAT, TOL, SEED = 1024, 512, 1e-13, 3


@pytest.mark.parametrize("k,trials", [(4, 100), (8, 50)])
def test_mixed_faults_converge_and_mostly_agree_with_oracle(k, trials):
    p = inputs.hill_problem(NLON, NLAT)
    ref = oracle.ftgcr(p.D, p.R, p.mu, k, TOL)
    with ftgcr.Solver(p.D, p.mu, k=k, tol=TOL, precision="mixed") as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        s.solve(R, x)
        clean = s.stats()
        # inner steps of the first refinement sweep: a mixed step t there is the
        # oracle's step t from the same start
        x.zero_()
        s1 = ftgcr.Solver(p.D, p.mu, k=k, tol=TOL, precision="mixed", max_outer=1)
        s1.solve(R, x)
        n1 = s1.stats()["steps"]
        s1.close()
        oracle.build()
        ctx = mp.get_context("spawn")
        with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            refs = dict((t, (d, c)) for t, d, c in pool.map(
                sweep_worker.oracle_mixed_counterpart, [(NLON, NLAT, k, TOL, SEED, t, n1) for t in range(trials)]))
        agree, worst = 0, 0.0
        for t in range(trials):
            f = inputs.sweep_flip(SEED, t, n1, NLON * NLAT, nbits=32)
            x.zero_()
            st = s.solve(R, x, faults=[f])
            info = s.stats()
            assert st == ftgcr.OK and info["converged"], (t, f, info)
            worst = max(worst, rel_err(x.cpu().numpy(), ref["x"]))
            agree += (info["faults_detected"] > 0) == refs[t][0]
    print(f"k={k}: {trials} flips, first sweep {n1} of {clean['steps']} inner steps, detection agreement "
          f"{agree}/{trials}, worst rel err {worst:.2e}")
    assert worst <= 1e-10
    assert agree >= 0.6 * trials
