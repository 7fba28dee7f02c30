"""FTGCR_FLAG_ZERO_GUESS: every solve starts from x = 0 and x is output only.
A flagged solve, whatever x holds on entry (here garbage, NaN included, on the
device and on the host), gives the result of the same solve from a zeroed x:
bitwise on the FP64 path (fault decisions included); on the mixed path the
first refinement round is skipped and the step counts and decisions are the
same, the solution equal to rounding of the norm of R.  Batches and the server
mix flagged and unflagged solves; R = 0 returns x = 0."""
import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("steps", "detect_steps", "faults_detected", "restarts", "converged", "outer")


def _run(p, precision, zero_guess, faults=(), rounds="auto", host=False, garbage=True, k=4):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=1e-10, precision=precision, rounds=rounds, zero_guess=zero_guess) as s:
        x = np.full(p.R.shape, np.nan) if garbage else np.zeros_like(p.R)
        if host:
            s.solve(p.R, x, faults=faults)
            return x, s.stats()
        R = torch.from_numpy(p.R).cuda()
        xt = torch.from_numpy(x).cuda()
        s.solve(R, xt, faults=faults)
        return xt.cpu().numpy(), s.stats()


@pytest.mark.parametrize("nlon,nlat,rhs,faults", [
    (64, 32, "random", [(5, "r", 700, 62)]),
    (512, 256, "flow", [(1, "x", 1234, 52), (4, "ap", 9000, 61)]),
    (1024, 512, "flow", ()),
])
@pytest.mark.parametrize("host", [False, True])
def test_fp64_zero_guess_is_bitwise_the_zeroed_solve(nlon, nlat, rhs, faults, host):
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=3)
    xa, sa = _run(p, "fp64", False, faults, host=host, garbage=False)
    xb, sb = _run(p, "fp64", True, faults, host=host)
    assert np.array_equal(xa, xb)
    for key in KEYS + ("res_final_true",):
        assert sa[key] == sb[key], key


@pytest.mark.parametrize("nlon,nlat,rounds", [(1024, 512, "auto"), (256, 128, "auto"), (1024, 64, "streamed"),
                                               (4096, 24, "split"), (100, 37, "auto")])
@pytest.mark.parametrize("host", [False, True])
def test_mixed_zero_guess_takes_the_same_steps(nlon, nlat, rounds, host):
    p = inputs.hill_problem(nlon, nlat, rhs="flow")
    xa, sa = _run(p, "mixed", False, rounds=rounds, host=host, garbage=False)
    xb, sb = _run(p, "mixed", True, rounds=rounds, host=host)
    for key in KEYS:
        assert sa[key] == sb[key], key
    assert rel_err(xb, xa) <= 1e-12
    assert sb["res_final_true"] <= 1e-10 * sb["norm_R"]


def test_mixed_zero_guess_with_faults_matches_the_zeroed_solve():
    p = inputs.hill_problem(256, 128, rhs="random", seed=9)
    faults = [(3, "r", 5000, 30), (7, "ap", 777, 29)]
    xa, sa = _run(p, "mixed", False, faults, garbage=False)
    xb, sb = _run(p, "mixed", True, faults)
    for key in KEYS:
        assert sa[key] == sb[key], key
    assert rel_err(xb, xa) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_rhs_with_zero_guess_returns_zero(precision):
    p = inputs.hill_problem(64, 32)
    p.R = np.zeros_like(p.R)
    x, s = _run(p, precision, True)
    assert s["converged"] and s["steps"] == 0
    assert np.array_equal(x, np.zeros_like(x))


def test_batch_and_server_mix_flagged_and_unflagged_solves():
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(120 + q)) for q, (n, m) in
             enumerate([(256, 128), (128, 64), (512, 256), (128, 64)])]
    flags = [True, False, True, True]
    alone = [_run(p, "mixed", z, garbage=z) for p, z in zip(probs, flags)]
    solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="mixed", zero_guess=z)
               for p, z in zip(probs, flags)]
    try:
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        xs = [torch.full_like(R, float("nan")) if z else torch.zeros_like(R) for R, z in zip(Rs, flags)]
        ftgcr.solve_batch(solvers, Rs, xs)
        torch.cuda.synchronize()
        for q, x in enumerate(xs):
            assert np.array_equal(x.cpu().numpy(), alone[q][0]), q
    finally:
        for s in solvers:
            s.close()
    with ftgcr.Server(max_slots=3, epoch_rounds=5) as srv:
        xh = [np.full(p.R.shape, np.nan) if z else np.zeros_like(p.R) for p, z in zip(probs, flags)]
        ts = [srv.submit(torch.from_numpy(p.D).cuda(), p.mu, p.R, x, precision="mixed", zero_guess=z)
              for p, x, z in zip(probs, xh, flags)]
        res = [srv.wait(t, timeout=60) for t in ts]
    for q, (st, ss) in enumerate(res):
        assert st == ftgcr.OK
        assert np.array_equal(xh[q], alone[q][0]), q


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refused_zero_guess_host_solve_returns_zero(precision):
    p = inputs.hill_problem(64, 32)
    R = p.R.copy()
    R[3, 5] = np.nan
    x = np.full(p.R.shape, 7.0)
    with ftgcr.Solver(p.D, p.mu, precision=precision, zero_guess=True) as s:
        with pytest.raises(ftgcr.FTGCRError) as ei:
            s.solve(R, x)
    assert ei.value.status == ftgcr.ERR_ARG
    assert np.array_equal(x, np.zeros_like(x))
