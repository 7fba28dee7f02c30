"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle:
operator bitwise, preconditioner to rounding, and whole FT-GCR(k) solves with
identical decisions (steps, detection steps, convergence) and solutions to
1e-10 relative error on the FP64 path."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import decisions, rel_err, rel_err_fault_trial

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def run(p, k=4, tol=1e-10, faults=(), precision="fp64", precond="line", x0=None, **kw):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision=precision, precond=precond, **kw) as s:
        R = cuda(p.R)
        x = cuda(x0) if x0 is not None else torch.zeros_like(R)
        st = s.solve(R, x, faults=list(faults))
        info = s.stats()
        torch.cuda.synchronize()
        return st, x.cpu().numpy(), info


PRECONDS = {"line": oracle.PRECOND_LINE, "jacobi": oracle.PRECOND_JACOBI, "identity": oracle.PRECOND_IDENTITY}


@pytest.mark.parametrize("nlon,nlat", [(64, 32), (40, 21), (3, 1), (100, 7), (1024, 512), (2048, 1024)])
def test_operator_is_bitwise_the_oracle(nlon, nlat):
    p = inputs.hill_problem(nlon, nlat, h0=0.15, centre=(0.5, 0.3))
    phi = inputs.uniform_pm1(17, (nlat, nlon))
    ref = oracle.apply_L(p.D, p.mu, phi)
    with ftgcr.Solver(p.D, p.mu) as s:
        out = torch.empty(nlat, nlon, dtype=torch.float64, device=DEV)
        s.apply_operator(cuda(phi), out)
        torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("precond", ["line", "jacobi", "identity"])
@pytest.mark.parametrize("nlon,nlat", [(64, 32), (40, 21), (3, 2), (1024, 512), (2048, 64), (33, 5)])
def test_preconditioner_matches_oracle(precond, nlon, nlat):
    p = inputs.hill_problem(nlon, nlat)
    r = inputs.uniform_pm1(23, (nlat, nlon))
    ref = oracle.solve_P(p.D, p.mu, r, PRECONDS[precond])
    with ftgcr.Solver(p.D, p.mu, precond=precond) as s:
        out = torch.empty(nlat, nlon, dtype=torch.float64, device=DEV)
        s.apply_precond(cuda(r), out)
        torch.cuda.synchronize()
    got = out.cpu().numpy()
    # the FP64 path runs the oracle's factorisation and substitution
    # operation for operation: bitwise equal
    assert np.array_equal(got, ref)


def test_config1_single_flip_at_step5():
    """64 x 32, k = 4, hill coefficients, seeded random RHS, tol 1e-10, one
    seeded flip in the residual at step 5."""
    p = inputs.hill_problem(64, 32, rhs="random", seed=1)
    N = p.nlon * p.nlat
    flip = inputs.single_flip(1, 5, "r", N)
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[flip])
    st, x, info = run(p, faults=[flip])
    assert st == ftgcr.OK
    assert decisions(info) == decisions(ref)
    assert info["faults_injected"] == ref["faults_injected"] == 1
    assert rel_err(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("nlon,nlat,k,precond,rhs", [
    (64, 32, 4, "line", "flow"), (64, 32, 1, "line", "random"), (64, 32, 8, "jacobi", "random"),
    (40, 21, 3, "line", "random"), (32, 16, 5, "identity", "random"), (512, 256, 4, "line", "flow"),
    (100, 7, 2, "line", "random"), (16, 1, 4, "line", "random"), (3, 2, 2, "jacobi", "random"),
    (1024, 512, 4, "line", "flow"), (1024, 512, 8, "line", "random"), (256, 128, 16, "line", "random"),
])
def test_fault_free_solve_matches_oracle(nlon, nlat, k, precond, rhs):
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=5)
    ref = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, precond=PRECONDS[precond])
    st, x, info = run(p, k=k, precond=precond)
    assert decisions(info) == decisions(ref)
    assert rel_err(x, ref["x"]) <= 1e-10
    assert info["res_final_true"] == pytest.approx(ref["res_true"], rel=1e-3, abs=1e-13 * np.sqrt(ref["nrm2_R"]))


@pytest.mark.parametrize("vec", ["x", "r", "p", "ap", "e"])
def test_fault_decisions_match_oracle_small_sweep(vec):
    p = inputs.hill_problem(128, 64)
    N = p.nlon * p.nlat
    ff = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10) as s:
        R = cuda(p.R)
        for trial in range(24):
            f = inputs.sweep_flip(1000, trial, ff["steps"], N, vecs=(vec,))
            ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[f])
            x = torch.zeros_like(R)
            s.solve(R, x, faults=[f])
            info = s.stats()
            assert decisions(info) == decisions(ref), (trial, f)
            assert info["faults_injected"] == ref["faults_injected"], (trial, f)
            # an undetected x / p flip: its entry holds scaled rounding
            e = rel_err_fault_trial(x.cpu().numpy(), ref["x"], f, info["faults_detected"] > 0)
            assert e <= 1e-10, (trial, f, e)


def test_first_step_flip_keeps_backup_clean():
    p = inputs.hill_problem(64, 32, rhs="random", seed=1)
    for f in [(1, "r", 17, 62), (1, "ap", 100, 62), (1, "x", 5, 62), (1, "p", 9, 61)]:
        ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[f])
        st, x, info = run(p, faults=[f])
        assert decisions(info) == decisions(ref), f
        assert rel_err(x, ref["x"]) <= 1e-10, f


def test_multiple_faults_in_one_plan():
    p = inputs.hill_problem(64, 32, rhs="random", seed=2)
    N = p.nlon * p.nlat
    plan = [(3, "r", 11, 62), (3, "e", 500, 40), (7, "ap", 1000, 62), (8, "x", 3, 63), (12, "r", 77, 62),
            (13, "p", 1200, 30)]
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=plan)
    st, x, info = run(p, faults=plan)
    assert decisions(info) == decisions(ref)
    assert info["faults_injected"] == ref["faults_injected"]
    assert rel_err(x, ref["x"]) <= 1e-10


def test_edge_cases():
    p = inputs.hill_problem(48, 24, rhs="random", seed=4)
    # zero right-hand side: x = 0 at once
    z = inputs.Problem(p.nlon, p.nlat, p.D, np.zeros_like(p.R), p.mu)
    st, x, info = run(z, x0=np.ones_like(p.R))
    assert st == ftgcr.OK and info["steps"] == 0 and np.all(x == 0)
    # exact initial guess: no step
    phi = inputs.uniform_pm1(3, p.R.shape)
    m = inputs.Problem(p.nlon, p.nlat, p.D, oracle.apply_L(p.D, p.mu, phi), p.mu)
    st, x, info = run(m, x0=phi)
    assert st == ftgcr.OK and info["steps"] == 0 and np.array_equal(x, phi)
    # step limit
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-14, max_steps=7)
    st, x, info = run(p, tol=1e-14, max_steps=7)
    assert st == ftgcr.NOT_CONVERGED and info["steps"] == 7 and not info["converged"]
    assert rel_err(x, ref["x"]) <= 1e-10


def test_host_pointers_match_device_pointers():
    p = inputs.hill_problem(96, 48, rhs="random", seed=6)
    st, xd, info = run(p)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10) as s:
        xh = np.zeros_like(p.R)
        st2 = s.solve(np.ascontiguousarray(p.R), xh)
    assert st2 == st and np.array_equal(xh, xd)


def test_invalid_arguments_are_rejected():
    p = inputs.hill_problem(32, 16)
    for bad in [dict(k=0), dict(k=17), dict(tol=0.0), dict(tol=-1.0)]:
        with pytest.raises(ftgcr.FTGCRError):
            ftgcr.Solver(p.D, p.mu, **bad)
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.Solver(np.ascontiguousarray(p.D[:, :2]), p.mu)
    D = p.D.copy()
    D[3, 3] = np.nan
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.Solver(D, p.mu)
    with ftgcr.Solver(p.D, p.mu) as s:
        R = cuda(p.R)
        x = torch.zeros_like(R)
        for f in [(0, "r", 1, 3), (2, "r", p.nlon * p.nlat, 3), (2, "r", 1, 64), (2, 7, 1, 3)]:
            with pytest.raises(ftgcr.FTGCRError):
                s.solve(R, x, faults=[f])


def test_non_finite_host_inputs_are_refused_and_the_handle_stays_usable():
    # host arrays are checked on the device after staging; the solve does not start
    p = inputs.hill_problem(64, 32, rhs="random", seed=12)
    for prec in ("fp64", "mixed"):
        with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision=prec) as s:
            xref = np.zeros_like(p.R)
            assert s.solve(np.ascontiguousarray(p.R), xref) == ftgcr.OK
            steps = s.stats()["steps"]
            bad_r = p.R.copy()
            bad_r[5, 7] = np.nan
            x = np.full_like(p.R, 0.5)
            with pytest.raises(ftgcr.FTGCRError) as ei:
                s.solve(bad_r, x)
            assert ei.value.status == ftgcr.ERR_ARG and np.all(x == 0.5)  # x comes back unchanged
            bad_x = np.zeros_like(p.R)
            bad_x[0, 0] = np.inf
            with pytest.raises(ftgcr.FTGCRError) as ei:
                s.solve(np.ascontiguousarray(p.R), bad_x)
            assert ei.value.status == ftgcr.ERR_ARG
            # the next solves, host and device, are unaffected
            x2 = np.zeros_like(p.R)
            assert s.solve(np.ascontiguousarray(p.R), x2) == ftgcr.OK and np.array_equal(x2, xref)
            assert s.stats()["steps"] == steps
            R = cuda(p.R)
            xd = torch.zeros_like(R)
            assert s.solve(R, xd) == ftgcr.OK and np.array_equal(xd.cpu().numpy(), xref)


def test_repeated_solves_on_one_handle_are_identical():
    p = inputs.hill_problem(128, 64, rhs="random", seed=9)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10) as s:
        R = cuda(p.R)
        xs = []
        for _ in range(3):
            x = torch.zeros_like(R)
            s.solve(R, x)
            xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[1], xs[2])
