"""GPU parity for the paper's data-loss fault events (Section 3), the
unprotected GCR(k) mode and the singular mu = 0 problem, through the C ABI.

FP64 path: decisions (steps, detection steps, convergence, events fired)
identical to the oracle's (the exit step of the long singular solves: in the
oracle's operation order), solution within 1e-10 relative.  Mixed path: converges to the oracle's
solution (rel <= 1e-10 at tol 1e-13) under data loss; batched solves with data
loss equal the same solves alone."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _events(seed, N, fracs, steps, nranks=12):
    g = inputs.SplitMix64(seed)
    return [(int(t), g.below(nranks), nranks, max(1, int(round(f * N))), g.next()) for t, f in zip(steps, fracs)]


def _gpu(p, k, tol, faults=(), losses=(), protect=True, precision="fp64", max_steps=0, mu=None, oracle_order=False):
    with ftgcr.Solver(p.D, p.mu if mu is None else mu, k=k, tol=tol, precision=precision, protect=protect,
                      max_steps=max_steps, oracle_order=oracle_order) as s:
        R = cuda(p.R)
        x = torch.zeros_like(R)
        st = s.solve(R, x, faults=faults, losses=losses)
        return st, x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("nlon,nlat,k,fracs,steps", [
    (128, 64, 5, [4e-6, 4e-4], [3, 7]),
    (128, 64, 5, [2e-3, 1e-2, 5e-2], [2, 5, 9]),
    (256, 128, 4, [0.2], [6]),
    (100, 37, 3, [1e-2, 1e-2], [4, 4]),
    (64, 32, 2, [5e-2], [1]),
])
def test_fp64_data_loss_matches_oracle(nlon, nlat, k, fracs, steps):
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=21)
    N = p.R.size
    ev = _events(nlon + nlat + k, N, fracs, steps)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, losses=[e + (64,) for e in ev])
    st, x, s = _gpu(p, k, 1e-10, losses=ev)
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"]
    assert s["converged"] == o["converged"] and s["loss_events"] == o["loss_events"]
    assert rel_err(x, o["x"]) <= 1e-10


def test_fp64_unprotected_matches_oracle():
    p = inputs.hill_problem(128, 64, rhs="random", seed=22)
    N = p.R.size
    faults = [(5, "r", 1000, 62), (8, "ap", 2000, 61)]
    ev = _events(5, N, [1e-2, 5e-2], [3, 10])
    o = oracle.ftgcr(p.D, p.R, p.mu, 5, 1e-10, faults=faults, losses=[e + (64,) for e in ev], protect=False,
                     max_steps=400)
    st, x, s = _gpu(p, 5, 1e-10, faults=faults, losses=ev, protect=False, max_steps=400)
    assert s["faults_detected"] == 0 and s["restarts"] == 0
    assert s["steps"] == o["steps"] and s["converged"] == o["converged"]
    if o["converged"]:
        assert rel_err(x, o["x"]) <= 1e-10
    # the same plan, protected, detects and replays
    st2, x2, s2 = _gpu(p, 5, 1e-10, faults=faults, losses=ev, max_steps=400)
    o2 = oracle.ftgcr(p.D, p.R, p.mu, 5, 1e-10, faults=faults, losses=[e + (64,) for e in ev], max_steps=400)
    assert s2["detect_steps"] == o2["detect_steps"] and s2["steps"] == o2["steps"]


@pytest.mark.parametrize("nlon,nlat,k", [(64, 32, 4), (128, 64, 6)])
@pytest.mark.parametrize("oracle_order", [True, False])
def test_fp64_mu_zero_matches_oracle(nlon, nlat, k, oracle_order):
    """Hundreds of slowly converging steps: in the oracle's operation order the
    exit step is the oracle's; by default (inner products summed by fma within
    each thread) it may move by a few percent (measured: 260 against 259 steps
    at 128 x 64, k = 6), with no detection and the same solution."""
    p = inputs.hill_problem(nlon, nlat, rhs="flow", mu_hat=0.0)
    R = p.R - p.R.mean()
    p.R = R
    o = oracle.ftgcr(p.D, R, 0.0, k, 1e-10)
    st, x, s = _gpu(p, k, 1e-10, mu=0.0, oracle_order=oracle_order)
    assert o["converged"] and s["converged"]
    assert s["detect_steps"] == o["detect_steps"] == []
    if oracle_order:
        assert s["steps"] == o["steps"]
    else:
        assert abs(s["steps"] - o["steps"]) <= 0.05 * o["steps"]
    assert rel_err(x - x.mean(), o["x"] - o["x"].mean()) <= 1e-10


def test_mixed_mu_zero_converges_to_the_oracle_solution():
    p = inputs.hill_problem(256, 128, rhs="flow", mu_hat=0.0)
    p.R = p.R - p.R.mean()
    o = oracle.ftgcr(p.D, p.R, 0.0, 4, 1e-12)
    st, x, s = _gpu(p, 4, 1e-12, precision="mixed", mu=0.0)
    assert st == ftgcr.OK and s["converged"]
    assert rel_err(x - x.mean(), o["x"] - o["x"].mean()) <= 1e-8


def test_mixed_data_loss_still_converges():
    p = inputs.hill_problem(256, 128, rhs="random", seed=23)
    N = p.R.size
    ref = oracle.ftgcr(p.D, p.R, p.mu, 5, 1e-13)
    for trial, fr in enumerate([4e-4, 1e-2, 5e-2, 0.2]):
        ev = _events(100 + trial, N, [fr, fr], [4, 11])
        st, x, s = _gpu(p, 5, 1e-13, losses=ev, precision="mixed")
        assert st == ftgcr.OK and s["converged"], (fr, s)
        assert rel_err(x, ref["x"]) <= 1e-10, fr


def test_batch_with_data_loss_equals_alone():
    probs = [inputs.hill_problem(n, n // 2, **inputs.random_hill(60 + n)) for n in (64, 128, 256)]
    evs = [_events(7 + q, p.R.size, [1e-2, 0.05], [3, 6]) for q, p in enumerate(probs)]
    for prec in ("fp64", "mixed"):
        alone = [_gpu(p, 4, 1e-10, losses=ev, precision=prec) for p, ev in zip(probs, evs)]
        solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision=prec) for p in probs]
        Rs = [cuda(p.R) for p in probs]
        xs = [torch.zeros_like(R) for R in Rs]
        ftgcr.solve_batch(solvers, Rs, xs, losses=evs)
        torch.cuda.synchronize()
        for q, s in enumerate(solvers):
            st = s.stats()
            assert np.array_equal(xs[q].cpu().numpy(), alone[q][1]), (prec, q)
            assert st["steps"] == alone[q][2]["steps"] and st["loss_events"] == alone[q][2]["loss_events"]
            s.close()


def test_invalid_loss_events_are_refused():
    p = inputs.hill_problem(64, 32)
    with ftgcr.Solver(p.D, p.mu) as s:
        R = cuda(p.R)
        for bad in [(0, 0, 4, 10, 1), (3, 4, 4, 10, 1), (3, 0, 0, 10, 1), (3, 0, 4, -1, 1)]:
            with pytest.raises(ftgcr.FTGCRError):
                s.solve(R, torch.zeros_like(R), losses=[bad])
