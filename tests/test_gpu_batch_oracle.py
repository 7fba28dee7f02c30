"""A batch in the shape of the 128-solve mix (uneven sizes up to 1024 x 512,
random hill centres, heights and widths, flow right-hand sides) with one
seeded bit flip, in ONE persistent mixed-precision launch, run eagerly and by
CUDA-graph replay: every result is compared with the FP64 oracle's solution
of its own problem (relative error <= 1e-10 at tol 1e-13), and with the same
handle solved alone (bitwise).  The oracle solves run in spawned workers
started before the first GPU call."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs
from tests import sweep_worker
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, K, SEED, NSOLVES = 1e-13, 4, 42, 12


def _sizes():
    sizes = inputs.batch_sizes(SEED, NSOLVES)
    if (1024, 512) not in sizes:
        sizes[0] = (1024, 512)
    return sizes


@pytest.fixture(scope="module")
def oracle_x():
    import oracle

    oracle.build()
    args = [(n, m, K, TOL, "flow", 1, SEED * 1000 + q) for q, (n, m) in enumerate(_sizes())]
    with mp.get_context("spawn").Pool(min(8, len(args))) as pool:
        return pool.map(sweep_worker.oracle_solution, args)


def test_batch_eager_and_graph_replay_match_the_oracle(oracle_x):
    sizes = _sizes()
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(SEED * 1000 + q)) for q, (n, m) in enumerate(sizes)]
    faults = [()] * len(probs)
    q1 = sizes.index((1024, 512))
    faults[q1] = [inputs.single_flip(SEED, 4, "r", sizes[q1][0] * sizes[q1][1], nbits=32)]
    solvers = [ftgcr.Solver(p.D, p.mu, k=K, tol=TOL, precision="mixed") for p in probs]
    try:
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        alone = []
        for s, R, f in zip(solvers, Rs, faults):
            x = torch.zeros_like(R)
            s.solve(R, x, faults=f)
            alone.append(x.clone())
        # eager batch
        xs = [torch.zeros_like(R) for R in Rs]
        ftgcr.solve_batch(solvers, Rs, xs, faults=faults)
        torch.cuda.synchronize()
        worst = 0.0
        for q, (s, x) in enumerate(zip(solvers, xs)):
            info = s.stats()
            assert info["converged"] and info["res_final_true"] <= TOL * info["norm_R"], (q, info)
            assert torch.equal(x, alone[q]), q
            xref, conv, _ = oracle_x[q]
            assert conv
            e = rel_err(x.cpu().numpy(), xref)
            worst = max(worst, e)
            assert e <= 1e-10, (q, sizes[q], e)
        assert solvers[q1].stats()["faults_injected"] == 1
        # the same launch captured into a CUDA graph and replayed twice
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ftgcr.solve_batch(solvers, Rs, xs, faults=faults, stream=side)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ftgcr.solve_batch(solvers, Rs, xs, faults=faults, stream=torch.cuda.current_stream())
        for _ in range(2):
            for x in xs:
                x.zero_()
            g.replay()
            torch.cuda.synchronize()
            for q, x in enumerate(xs):
                assert torch.equal(x, alone[q]), q
                assert rel_err(x.cpu().numpy(), oracle_x[q][0]) <= 1e-10, q
        print(f"{len(probs)} solves, sizes {sorted(set(sizes))}: worst rel err vs oracle {worst:.2e}")
    finally:
        for s in solvers:
            s.close()
