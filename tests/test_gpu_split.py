"""Split rounds (mixed path): each step's tiles first form e on their own rows,
then, after a grid barrier, L(e) and the dots from e with its halo rows.
Forced on small grids (ragged bands, rows not a multiple of four, a single
latitude row per band, several directions) the solve matches the FP64 oracle
as the one-pass layout does (rel <= 1e-10 at tol 1e-13); under faults and
data loss it still converges to the oracle's solution; chosen automatically
where shared memory cuts bands below three rows, and it lets rows twice as
wide as the one-pass layout allows be solved; batched and served split
solves equal the same solves alone, bitwise."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _solve(p, k, tol, rounds, faults=(), losses=(), tiles=0):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision="mixed", rounds=rounds, tiles=tiles) as s:
        R = cuda(p.R)
        x = torch.zeros_like(R)
        st = s.solve(R, x, faults=faults, losses=losses)
        return st, x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("nlon,nlat,k,rhs,tiles", [
    (128, 64, 4, "flow", 0), (100, 37, 3, "random", 0), (130, 40, 5, "random", 0), (64, 3, 2, "random", 0),
    (256, 128, 8, "flow", 16), (512, 96, 4, "random", 0), (2048, 16, 4, "random", 0),
])
def test_split_rounds_match_fp64_oracle(nlon, nlat, k, rhs, tiles):
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=41)
    tol = 1e-12 if nlon >= 2048 else 1e-13  # wide rows: attainable accuracy about 1e-12
    ref = oracle.ftgcr(p.D, p.R, p.mu, k, tol)
    assert ref["converged"]
    st, x, s = _solve(p, k, tol, "split", tiles=tiles)
    assert st == ftgcr.OK and s["converged"] and s["split_rounds"], s
    assert s["res_final_true"] <= tol * s["norm_R"]
    assert rel_err(x, ref["x"]) <= (1e-7 if nlon >= 2048 else 1e-10)
    # the one-pass layout of the same problem agrees to the same accuracy
    st2, x2, s2 = _solve(p, k, tol, "fused", tiles=tiles)
    assert st2 == ftgcr.OK and not s2["split_rounds"]
    assert rel_err(x, x2) <= (1e-7 if nlon >= 2048 else 1e-10)


def test_split_rounds_under_faults_and_data_loss_converge_to_the_oracle():
    p = inputs.hill_problem(256, 128, rhs="random", seed=42)
    N = p.R.size
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-13)
    g = inputs.SplitMix64(9)
    plans = [
        ([(3, "r", 1000, 30), (5, "e", 20000, 29), (7, "ap", 777, 30), (9, "x", 12345, 30), (11, "p", 500, 30)], ()),
        ((), [(4, g.below(8), 8, int(0.01 * N), g.next()), (9, g.below(8), 8, int(0.05 * N), g.next())]),
        ([(2, "e", 5, 31)], [(6, 3, 8, int(0.2 * N), g.next())]),
    ]
    for faults, losses in plans:
        st, x, s = _solve(p, 4, 1e-13, "split", faults=faults, losses=losses)
        assert st == ftgcr.OK and s["converged"] and s["split_rounds"], (faults, losses, s)
        assert rel_err(x, ref["x"]) <= 1e-10
        if losses:
            assert s["loss_events"] == len(losses)


def test_split_and_fused_see_the_same_faults():
    # the same plan fires the same flips in both layouts (decisions may differ
    # only through rounding of the FP32 inner vectors)
    p = inputs.hill_problem(128, 64, rhs="random", seed=43)
    faults = [(4, "r", 3000, 30), (8, "ap", 100, 30)]
    a = _solve(p, 4, 1e-10, "split", faults=faults)[2]
    b = _solve(p, 4, 1e-10, "fused", faults=faults)[2]
    assert a["faults_injected"] == b["faults_injected"] == 2
    assert a["faults_detected"] >= 1 and b["faults_detected"] >= 1


def test_automatic_choice_and_rows_beyond_the_one_pass_limit():
    p = inputs.hill_problem(1024, 512)
    assert not _solve(p, 4, 1e-10, "auto")[2]["split_rounds"]  # bands of 4 rows: one pass
    wide = inputs.hill_problem(4096, 304, rhs="random", seed=44)  # bands cut to 1 row by shared memory
    with ftgcr.Solver(wide.D, wide.mu, precision="mixed") as s:
        R = cuda(wide.R)
        x = torch.zeros_like(R)
        assert s.solve(R, x) == ftgcr.OK
        info = s.stats()
    assert info["split_rounds"] and info["converged"] and info["tiles"] < 304
    p8 = inputs.hill_problem(8192, 8, rhs="random", seed=45)
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.Solver(p8.D, p8.mu, precision="mixed", rounds="fused")
    ref = oracle.ftgcr(p8.D, p8.R, p8.mu, 4, 1e-12)
    st, x, s = _solve(p8, 4, 1e-10, "auto")
    assert st == ftgcr.OK and s["split_rounds"] and s["res_final_true"] <= 1e-10 * s["norm_R"]
    assert rel_err(x, ref["x"]) <= 1e-7


def test_batched_split_solves_equal_alone():
    # (2048, 16) in one pass: its 1-row bands would take warp groups in a split
    # round's first pass; one-pass rounds never do, in either kernel instance
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(70 + n))
             for n, m in ((128, 64), (256, 96), (64, 32), (2048, 16), (512, 8))]
    rounds = ["split", "fused", "split", "fused", "split"]
    alone = [_solve(p, 4, 1e-10, r) for p, r in zip(probs, rounds)]
    solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="mixed", rounds=r) for p, r in zip(probs, rounds)]
    Rs = [cuda(p.R) for p in probs]
    xs = [torch.zeros_like(R) for R in Rs]
    ftgcr.solve_batch(solvers, Rs, xs)
    torch.cuda.synchronize()
    for q, s in enumerate(solvers):
        assert np.array_equal(xs[q].cpu().numpy(), alone[q][1]), q
        assert s.stats()["steps"] == alone[q][2]["steps"]
        s.close()


def test_served_split_solves_equal_alone():
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(80 + n)) for n, m in ((128, 64), (256, 128), (96, 48))]
    with ftgcr.Server(max_slots=4, epoch_rounds=7) as srv:
        xs = [np.zeros_like(p.R) for p in probs]
        ts = [srv.submit(p.D, p.mu, p.R, x, precision="mixed", rounds="split") for p, x in zip(probs, xs)]
        res = [srv.wait(t, timeout=60) for t in ts]
    # solo runs with the bands the server reported
    alone = [_solve(p, 4, 1e-10, "split", tiles=ss["tiles"]) for p, (_, ss) in zip(probs, res)]
    for q, (st, ss) in enumerate(res):
        assert st == ftgcr.OK and ss["split_rounds"]
        assert np.array_equal(xs[q], alone[q][1]) and ss["steps"] == alone[q][2]["steps"], q
