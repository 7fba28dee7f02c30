"""Batched solves (ftgcr_solve_batch: one persistent launch for many
independent problems of different sizes): every result, counters included,
is bitwise the one the same handle produces alone."""
import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems(sizes, seed):
    out = []
    for q, (nlon, nlat) in enumerate(sizes):
        p = inputs.hill_problem(nlon, nlat, **inputs.random_hill(seed + q))
        out.append(p)
    return out


def _run_both(problems, precision, k, faults):
    solvers = [ftgcr.Solver(p.D, p.mu, k=k, tol=1e-10, precision=precision) for p in problems]
    R = [torch.from_numpy(p.R).cuda() for p in problems]
    alone, alone_info = [], []
    for s, r, f in zip(solvers, R, faults):
        x = torch.zeros_like(r)
        s.solve(r, x, faults=f)
        alone.append(x.cpu().numpy())
        alone_info.append(s.stats())
    xs = [torch.zeros_like(r) for r in R]
    ftgcr.solve_batch(solvers, R, xs, faults=faults)
    torch.cuda.synchronize()
    batch_info = [s.stats() for s in solvers]
    for s in solvers:
        s.close()
    return alone, alone_info, [x.cpu().numpy() for x in xs], batch_info


KEYS = ("steps", "cycles", "restarts", "faults_injected", "faults_detected", "outer", "converged", "detect_steps",
        "res_final_rec", "res_final_true", "status")


@pytest.mark.parametrize("precision,k", [("fp64", 4), ("mixed", 4), ("mixed", 8)])
def test_batch_results_are_bitwise_the_solo_results(precision, k):
    sizes = [(128, 64), (64, 32), (256, 128), (40, 21), (512, 256), (100, 7), (1024, 512), (256, 128)]
    problems = _problems(sizes, 31)
    nb = 32 if precision == "mixed" else 64
    faults = [()] * len(problems)
    faults[1] = [(3, "r", 100, nb - 2)]
    faults[4] = [(5, "ap", 777, nb - 2), (9, "e", 12345, 20)]
    alone, ai, batch, bi = _run_both(problems, precision, k, faults)
    for q in range(len(problems)):
        assert ai[q]["converged"], (q, ai[q])
        assert np.array_equal(alone[q], batch[q]), q
        for key in KEYS:
            assert ai[q][key] == bi[q][key], (q, key, ai[q][key], bi[q][key])


def test_batch_rejects_mixed_precisions_and_duplicates():
    p = inputs.hill_problem(32, 16)
    a = ftgcr.Solver(p.D, p.mu, precision="fp64")
    b = ftgcr.Solver(p.D, p.mu, precision="mixed")
    R = torch.from_numpy(p.R).cuda()
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.solve_batch([a, b], [R, R], [torch.zeros_like(R), torch.zeros_like(R)])
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.solve_batch([a, a], [R, R], [torch.zeros_like(R), torch.zeros_like(R)])
    a.close()
    b.close()
