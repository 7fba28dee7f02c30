"""Long, slowly converging FP64 solves: the singular mu = 0 hill problem
(Section 3's pure Poisson form) takes hundreds of steps.

- With FTGCR_FLAG_ORACLE_ORDER every inner product is summed compensated and
  every row solved in the oracle's operation order, and the solve takes the
  oracle's decisions exactly: the same step count, no detections, the same
  solution (rel <= 1e-10, bitwise in practice).
- By default each thread sums its products by fma and rows of 256+ columns
  take the chunked scan: the same arithmetic rounded differently.  The
  solution still matches the oracle to 1e-10 and nothing is detected, but the
  exit may come a few percent of the steps earlier or later (measured with
  the chunked scan alone: 484 against 470 steps for k = 6 at 256 x 128).
- Fault decisions under single flips stay the oracle's in either mode."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mu0(nlon, nlat):
    p = inputs.hill_problem(nlon, nlat, rhs="flow", mu_hat=0.0)
    return p, p.R - p.R.mean()


def _gpu(p, R, mu, k, oracle_order, faults=(), max_steps=20000, tiles=0):
    with ftgcr.Solver(p.D, mu, k=k, tol=1e-10, precision="fp64", max_steps=max_steps, tiles=tiles,
                      oracle_order=oracle_order) as s:
        Rt = torch.from_numpy(np.ascontiguousarray(R)).cuda()
        x = torch.zeros_like(Rt)
        s.solve(Rt, x, faults=faults)
        return x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("nlon,nlat,k", [(256, 128, 6), (256, 128, 4), (320, 64, 4), (128, 64, 4)])
def test_oracle_order_takes_the_oracles_decisions_in_long_singular_solves(nlon, nlat, k):
    p, R = _mu0(nlon, nlat)
    o = oracle.ftgcr(p.D, R, 0.0, k, 1e-10, max_steps=20000)
    x, s = _gpu(p, R, 0.0, k, True)
    assert o["converged"] and s["converged"]
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"] == []
    assert rel_err(x - x.mean(), o["x"] - o["x"].mean()) <= 1e-10


@pytest.mark.parametrize("nlon,nlat,k", [(256, 128, 6), (128, 64, 4)])
def test_default_order_keeps_the_solution_and_no_detection_in_long_singular_solves(nlon, nlat, k):
    p, R = _mu0(nlon, nlat)
    o = oracle.ftgcr(p.D, R, 0.0, k, 1e-10, max_steps=20000)
    x, s = _gpu(p, R, 0.0, k, False)
    assert o["converged"] and s["converged"] and s["detect_steps"] == []
    assert abs(s["steps"] - o["steps"]) <= 0.05 * o["steps"]
    assert rel_err(x - x.mean(), o["x"] - o["x"].mean()) <= 1e-10


@pytest.mark.parametrize("oracle_order", [True, False])
@pytest.mark.parametrize("nlon,nlat,tiles", [(512, 256, 0), (2048, 48, 6)])  # staged; factors in global memory
def test_fault_decisions_match_in_either_mode(nlon, nlat, tiles, oracle_order):
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=44)
    N = p.R.size
    faults = [(4, "r", N // 3 + 7, 62), (9, "ap", N // 2 + 1, 61)]
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=faults)
    x, s = _gpu(p, p.R, p.mu, 4, oracle_order, faults=faults, max_steps=0, tiles=tiles)
    assert s["global_factors"] == (tiles > 0)
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"]
    assert s["faults_detected"] == o["faults_detected"] and s["converged"] == o["converged"]
    assert rel_err(x, o["x"]) <= 1e-10


def test_oracle_order_is_refused_on_the_mixed_path():
    p = inputs.hill_problem(64, 32)
    for pc in ("line", "jacobi"):
        with pytest.raises(ftgcr.FTGCRError):
            ftgcr.Solver(p.D, p.mu, precision="mixed", precond=pc, oracle_order=True)


@pytest.mark.parametrize("precond", ["jacobi", "identity"])
def test_oracle_order_with_other_preconditioners_takes_the_oracles_steps(precond):
    p = inputs.hill_problem(96, 48, rhs="random", seed=5)
    pc = {"jacobi": oracle.PRECOND_JACOBI, "identity": oracle.PRECOND_IDENTITY}[precond]
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, precond=pc, max_steps=20000)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="fp64", precond=precond, oracle_order=True) as s:
        Rt = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(Rt)
        s.solve(Rt, x)
        st = s.stats()
    assert o["converged"] and st["converged"] and st["steps"] == o["steps"]
    assert rel_err(x.cpu().numpy(), o["x"]) <= 1e-10


@pytest.mark.parametrize("nlon,nlat,k,flip", [(128, 64, 4, None), (100, 37, 3, (5, "r", 1234, 60)),
                                              (64, 32, 8, (3, "p", 700, 52))])
def test_oracle_order_is_bitwise_the_oracle_on_rows_under_256_columns(nlon, nlat, k, flip):
    """In the oracle's operation order (compensated sums, the oracle's stencil
    form, serial row solves) an FP64 solve on rows under 256 columns takes the
    oracle's arithmetic step by step: the same decisions and the same solution
    bit for bit, with or without a flip."""
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=17)
    faults = [flip] if flip else []
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, faults=faults)
    x, s = _gpu(p, p.R, p.mu, k, True, faults=faults, max_steps=0)
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"]
    assert np.array_equal(x, o["x"])


def test_batch_mixing_both_orders_equals_each_solve_alone():
    """One launch over FP64 solves in the default order and in the oracle's
    order (each solve carries its own flag): every result, the step count
    included, is bitwise the same solve alone, and those in the oracle's
    order are bitwise the oracle's."""
    probs = [inputs.hill_problem(n, m, rhs="random", seed=60 + i) for i, (n, m) in
             enumerate([(128, 64), (96, 48), (300, 40), (128, 64)])]
    orders = [True, False, True, False]
    solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="fp64", oracle_order=o) for p, o in zip(probs, orders)]
    try:
        R = [torch.from_numpy(p.R).cuda() for p in probs]
        alone, steps = [], []
        for s, r in zip(solvers, R):
            x = torch.zeros_like(r)
            s.solve(r, x)
            alone.append(x.cpu().numpy())
            steps.append(s.stats()["steps"])
        xs = [torch.zeros_like(r) for r in R]
        ftgcr.solve_batch(solvers, R, xs)
        torch.cuda.synchronize()
        for s, x, a, st in zip(solvers, xs, alone, steps):
            assert np.array_equal(x.cpu().numpy(), a) and s.stats()["steps"] == st
    finally:
        for s in solvers:
            s.close()
    for p, o, a in zip(probs, orders, alone):
        if o and p.nlon < 256:
            assert np.array_equal(a, oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)["x"])
