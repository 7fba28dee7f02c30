"""Mixed-precision path (FP32 inner FT-GCR vectors, stencil, preconditioner
and axpys; FP64 inner products, norm test and outer refinement residual)
against the FP64 oracle: relative solution error <= 1e-10 when both solve to
a tolerance well below it."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


@pytest.mark.parametrize("nlon,nlat,k,rhs", [
    (1024, 512, 4, "flow"), (1024, 512, 8, "flow"), (1024, 512, 4, "random"),
    (64, 32, 4, "random"), (40, 21, 3, "random"), (256, 128, 8, "flow"), (16, 1, 2, "random"),
])
def test_mixed_matches_fp64_oracle(nlon, nlat, k, rhs):
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=3)
    ref = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-13)
    assert ref["converged"]
    with ftgcr.Solver(p.D, p.mu, k=k, tol=1e-13, precision="mixed") as s:
        R = cuda(p.R)
        x = torch.zeros_like(R)
        st = s.solve(R, x)
        info = s.stats()
    assert st == ftgcr.OK and info["converged"], info
    assert info["res_final_true"] <= 1e-13 * info["norm_R"]
    assert rel_err(x.cpu().numpy(), ref["x"]) <= 1e-10
    assert info["outer"] >= 2  # FP32 inner solves alone cannot reach 1e-13


def test_mixed_at_config_tolerance():
    # the benchmark configuration: 1024 x 512, k = 4, tol 1e-10
    p = inputs.hill_problem(1024, 512)
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="mixed") as s:
        R = cuda(p.R)
        x = torch.zeros_like(R)
        s.solve(R, x)
        info = s.stats()
    assert info["converged"] and info["res_final_true"] <= 1e-10 * info["norm_R"]
    # both residuals are below 1e-10 ||R||; the errors differ by at most cond * tol
    assert rel_err(x.cpu().numpy(), ref["x"]) <= 1e-8


def test_mixed_with_inner_faults_still_converges():
    p = inputs.hill_problem(256, 128, rhs="random", seed=4)
    N = p.nlon * p.nlat
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-13)
    det = 0
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-13, precision="mixed") as s:
        R = cuda(p.R)
        for trial in range(30):
            f = inputs.sweep_flip(77, trial, 30, N, nbits=32, vecs=("x", "r", "p", "ap", "e"))
            x = torch.zeros_like(R)
            st = s.solve(R, x, faults=[f])
            info = s.stats()
            det += info["faults_detected"]
            assert st == ftgcr.OK and info["converged"], (trial, f, info)
            assert rel_err(x.cpu().numpy(), ref["x"]) <= 1e-10, (trial, f)
    assert det > 0
