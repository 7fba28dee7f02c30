"""ftgcr_solve_host_async: the host-array solve enqueued without waiting.
Through the C ABI, with pinned host arrays:
  * one solve gives bitwise the solution, step count and status of the
    blocking ftgcr_solve on the same problem;
  * solves of two handles alternating on two streams (copies of one
    overlapping the other's kernel) give bitwise each one's sequential result;
  * a NaN in a host right-hand side reports FTGCR_ERR_ARG through
    ftgcr_stats and leaves x as it was, and the handle solves normally after;
  * a device rhs with a host x works too."""
import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pinned(a):
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_async_equals_blocking_solve(precision):
    p = inputs.hill_problem(256, 128, rhs="random", seed=41)
    flip = [(5, "r", 999, 62 if precision == "fp64" else 30)]  # FP32 inner vectors: bits 0..31
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision=precision) as s:
        R, x = pinned(p.R), pinned(np.zeros_like(p.R))
        st_ref = s.solve(R, x, faults=flip)
        x_ref, info_ref = x.clone(), s.stats()
        x.zero_()
        stream = torch.cuda.Stream()
        s.solve_host_async(R, x, faults=flip, stream=stream)
        stream.synchronize()
        info = s.stats()
        assert info["status"] == st_ref == ftgcr.OK
        assert info["steps"] == info_ref["steps"] and info["detect_steps"] == info_ref["detect_steps"]
        assert torch.equal(x, x_ref)


def test_two_handles_pipelined_on_two_streams_equal_sequential():
    probs = [inputs.hill_problem(512, 256, **inputs.random_hill(q)) for q in range(4)]
    solvers = [ftgcr.Solver(probs[0].D, probs[0].mu, k=4, tol=1e-10, precision="mixed") for _ in range(2)]
    try:
        Rs = [pinned(p.R) for p in probs]
        ref = []
        for q, p in enumerate(probs):  # sequential, blocking
            s = solvers[q % 2]
            s.set_coeffs(torch.from_numpy(p.D).cuda())
            x = pinned(np.zeros_like(p.R))
            assert s.solve(Rs[q], x) == ftgcr.OK
            ref.append(x.clone())
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        Ds = [torch.from_numpy(p.D).cuda() for p in probs]
        xs = [pinned(np.zeros_like(p.R)) for p in probs]
        for q in range(4):
            b = q % 2
            if q >= 2:
                streams[b].synchronize()  # the handle's previous solve has ended
                assert solvers[b].stats()["status"] == ftgcr.OK
            solvers[b].set_coeffs(Ds[q], stream=streams[b])
            solvers[b].solve_host_async(Rs[q], xs[q], stream=streams[b])
        for b in range(2):
            streams[b].synchronize()
            assert solvers[b].stats()["status"] == ftgcr.OK
        for q in range(4):
            assert torch.equal(xs[q], ref[q]), q
    finally:
        for s in solvers:
            s.close()


def test_nonfinite_host_rhs_reports_err_arg_and_keeps_x():
    p = inputs.hill_problem(128, 64, rhs="random", seed=43)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10) as s:
        bad = p.R.copy()
        bad[7] = np.nan
        R, x = pinned(bad), pinned(np.full_like(p.R, 0.25))
        s.solve_host_async(R, x)
        torch.cuda.synchronize()
        assert s.stats()["status"] == ftgcr.ERR_ARG
        assert torch.all(x == 0.25)
        R.copy_(torch.from_numpy(p.R))
        x.zero_()
        s.solve_host_async(R, x)
        torch.cuda.synchronize()
        assert s.stats()["status"] == ftgcr.OK and torch.isfinite(x).all()


def test_device_rhs_host_x():
    p = inputs.hill_problem(128, 64, rhs="random", seed=44)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10) as s:
        Rd = torch.from_numpy(p.R).cuda()
        x_ref = torch.zeros_like(Rd)
        s.solve(Rd, x_ref)
        x = pinned(np.zeros_like(p.R))
        s.solve_host_async(Rd, x)
        torch.cuda.synchronize()
        assert s.stats()["status"] == ftgcr.OK
        assert torch.equal(x, x_ref.cpu())
