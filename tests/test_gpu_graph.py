"""A solve enqueued with ftgcr_solve_async can be captured into a CUDA graph
and replayed: the begin kernel, the cooperative persistent launch and the
copies of the result record are all stream-ordered and allocate nothing.
Every replay gives bitwise the eager solve's solution and counters.  A batch
(ftgcr_solve_batch, stream-ordered allocations and a kernel-filled solve
table) replays the same way."""
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_replays_from_a_cuda_graph(precision):
    p = inputs.hill_problem(256, 128, **inputs.random_hill(5))
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision=precision) as s:
        R = torch.from_numpy(p.R).cuda()
        x_ref = torch.zeros_like(R)
        s.solve(R, x_ref)
        ref = s.stats()
        x = torch.zeros_like(R)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # warm-up outside capture, as CUDA graphs want
            s.solve_async(R, x, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            s.solve_async(R, x, stream=torch.cuda.current_stream())
        for _ in range(3):
            x.zero_()
            g.replay()
            torch.cuda.synchronize()
            st = s.stats()
            assert torch.equal(x, x_ref)
            assert st["steps"] == ref["steps"] and st["converged"] and st["res_final_true"] == ref["res_final_true"]


def test_batch_replays_from_a_cuda_graph():
    """A batch of uneven solves in one persistent launch (ftgcr_solve_batch),
    captured once and replayed: every replay gives each solve's eager result."""
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(90 + n)) for n, m in ((64, 32), (256, 128), (128, 64))]
    solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="mixed") for p in probs]
    try:
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        refs = []
        for s, R in zip(solvers, Rs):
            x = torch.zeros_like(R)
            s.solve(R, x)
            refs.append((x, s.stats()["steps"]))
        xs = [torch.zeros_like(R) for R in Rs]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ftgcr.solve_batch(solvers, Rs, xs, stream=side)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ftgcr.solve_batch(solvers, Rs, xs, stream=torch.cuda.current_stream())
        for _ in range(3):
            for x in xs:
                x.zero_()
            g.replay()
            torch.cuda.synchronize()
            for s, x, (xr, steps) in zip(solvers, xs, refs):
                assert torch.equal(x, xr)
                assert s.stats()["steps"] == steps
    finally:
        for s in solvers:
            s.close()
