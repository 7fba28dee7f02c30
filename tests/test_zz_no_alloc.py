"""ftgcr_solve_noalloc: the FP64 solve for callers that cannot allocate device
memory when they solve (a process whose device memory belongs entirely to
another allocator, or code that must not fail with out-of-memory mid-run).
Its scratch is a static device array inside the library; the call blocks and
stages small records through host memory.  This test checks that
  * two calls in a row, through the C ABI, each give the solution of the
    ordinary allocating entry point (ftgcr_solve) to the FP64 tolerance the
    other tests use (1e-10 relative), with the same step count;
  * a repeated call leaves the device's free memory unchanged;
  * a result does not depend on the sizes of the calls before it;
  * a fresh process that has created no handle (so nothing has raised the
    per-thread stack limit) solves as well;
  * sizes beyond the stated maximum are rejected with an error.
Collected last (file name) so that a failure here cannot hide another test's."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(p, k, tol):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol) as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st = s.solve(R, x)
        return st, x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("nlon,nlat,k,rhs", [(128, 64, 4, "flow"), (100, 37, 3, "random")])
def test_noalloc_matches_allocating_solve_twice(nlon, nlat, k, rhs):
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=12)
    st_ref, x_ref, info_ref = _reference(p, k, 1e-10)
    D = torch.from_numpy(p.D).cuda()
    R = torch.from_numpy(p.R).cuda()
    free_after_first = None
    for call in range(2):
        x = torch.zeros_like(R)
        torch.cuda.synchronize()
        st, info = ftgcr.solve_noalloc(D, p.mu, R, x, k=k, tol=1e-10)
        torch.cuda.synchronize()
        if call == 0:
            free_after_first = torch.cuda.mem_get_info()[0]
        else:
            assert torch.cuda.mem_get_info()[0] == free_after_first
        assert st == st_ref == ftgcr.OK
        assert info["steps"] == info_ref["steps"] and info["converged"]
        assert rel_err(x.cpu().numpy(), x_ref) <= 1e-10


def test_noalloc_result_does_not_depend_on_the_previous_call_sizes():
    # the array keeps the last call's contents, laid out for that call's sizes
    probs = [inputs.hill_problem(n, m, rhs="random", seed=n + m) for n, m in ((128, 64), (40, 21), (96, 48))]
    refs = [_reference(p, 4, 1e-10) for p in probs]
    for q in (0, 1, 2, 1, 0, 2):
        p = probs[q]
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st, info = ftgcr.solve_noalloc(torch.from_numpy(p.D).cuda(), p.mu, R, x, k=4, tol=1e-10)
        assert st == ftgcr.OK and info["steps"] == refs[q][2]["steps"]
        assert rel_err(x.cpu().numpy(), refs[q][1]) <= 1e-10


def test_noalloc_rejects_sizes_beyond_its_maximum():
    for nlon, nlat, k in [(256, 128, 4), (128, 64, 5)]:  # 32768 points > 16384; k > 4
        p = inputs.hill_problem(nlon, nlat)
        D = torch.from_numpy(p.D).cuda()
        R = torch.from_numpy(p.R).cuda()
        with pytest.raises(ftgcr.FTGCRError) as ei:
            ftgcr.solve_noalloc(D, p.mu, R, torch.zeros_like(R), k=k)
        assert ei.value.status == ftgcr.ERR_ARG
    assert ftgcr.NOALLOC_MAX_POINTS == 16384 and ftgcr.NOALLOC_MAX_K == 4


_FRESH = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2103_07210_gb300 import ftgcr, inputs
p = inputs.hill_problem(128, 64, rhs="random", seed=21)
D = torch.from_numpy(p.D).cuda()
R = torch.from_numpy(p.R).cuda()
xs = []
for call in range(2):
    x = torch.zeros_like(R)
    st, info = ftgcr.solve_noalloc(D, p.mu, R, x, k=4, tol=1e-10)
    assert st == ftgcr.OK and info["converged"], (st, info)
    xs.append((x.cpu().numpy(), info["steps"]))
np.save(sys.argv[2], np.stack([xs[0][0], xs[1][0]]))
print(xs[0][1], xs[1][1])
"""


def test_noalloc_in_a_fresh_process_before_any_handle(tmp_path):
    # no ftgcr_create has run in the child, so the stack limit is CUDA's default
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x.npy")
    r = subprocess.run([sys.executable, "-c", _FRESH, root, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    steps = [int(v) for v in r.stdout.split()[-2:]]
    p = inputs.hill_problem(128, 64, rhs="random", seed=21)
    st_ref, x_ref, info_ref = _reference(p, 4, 1e-10)
    xs = np.load(out)
    for q in range(2):
        assert steps[q] == info_ref["steps"]
        assert rel_err(xs[q], x_ref) <= 1e-10
