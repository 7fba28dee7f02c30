"""Mixed-precision path on the HBM-resident grids (2048 x 1024 and
4096 x 2048, whose working sets exceed the 129 MB L2) against the FP64 oracle:
solution relative error <= 1e-10 when both solve to tol 1e-13.  These are the
grids the bench times for its HBM roofline, in the layouts ftgcr_create picks
for them (one-pass rounds at 2048 columns, split rounds at 4096).  The oracle
solves run in spawned worker processes, started before the first GPU call."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs
from tests import sweep_worker
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13
CASES = [(2048, 1024, 4, "flow"), (2048, 1024, 8, "random"), (4096, 2048, 4, "flow")]


@pytest.fixture(scope="module")
def oracle_x():
    import oracle

    oracle.build()
    args = [(n, m, k, TOL, rhs, 3, None) for n, m, k, rhs in CASES]
    with mp.get_context("spawn").Pool(len(args)) as pool:
        res = pool.map(sweep_worker.oracle_solution, args)
    return {c: r for c, r in zip(CASES, res)}


@pytest.mark.parametrize("case", CASES, ids=[f"{n}x{m}_k{k}_{r}" for n, m, k, r in CASES])
def test_mixed_large_grid_matches_fp64_oracle(oracle_x, case):
    nlon, nlat, k, rhs = case
    xref, conv, _ = oracle_x[case]
    assert conv
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=3)
    with ftgcr.Solver(p.D, p.mu, k=k, tol=TOL, precision="mixed") as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st = s.solve(R, x)
        info = s.stats()
    assert st == ftgcr.OK and info["converged"], info
    assert info["res_final_true"] <= TOL * info["norm_R"]
    err = rel_err(x.cpu().numpy(), xref)
    print(f"{nlon}x{nlat} k={k} {rhs}: rel err vs oracle {err:.2e}, {info['steps']} inner steps, "
          f"{info['outer']} sweeps, tiles {info['tiles']}")
    assert err <= 1e-10
