"""Wide latitude rows (FP64 2048 x 32; mixed 4096 x 16), whose staged rows and
line-solve constants fill shared memory so that each band holds a single
row: the same results as the oracle (FP64: identical decisions, solution
rel <= 1e-10; mixed, one-pass rounds: converged at tol 1e-10 with a true residual below it,
solution within 1e-7 of the oracle's at tol 1e-12 -- these strongly
anisotropic grids keep the true residual of any solve near 1e-12 relative, so
the mixed path's FP64 refinement cannot be asked for 1e-13 here).  FP64 solves
whose staged factors would thin the bands below what the SM count gives (or
not fit at all) read the factors from global memory: the same decisions and
solution as the oracle.  Rows too wide for one band on chip are refused at
creation."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(p, k, tol, precision, faults=(), tiles=0):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision=precision, tiles=tiles) as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st = s.solve(R, x, faults=faults)
        return st, x.cpu().numpy(), s.stats()


def test_fp64_wide_rows_match_oracle():
    p = inputs.hill_problem(2048, 32, rhs="random", seed=31)
    faults = [(4, "r", 40000, 62)]
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=faults)
    st, x, s = _solve(p, 4, 1e-10, "fp64", faults)
    assert s["tiles"] == 32 and not s["global_factors"]
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"] and s["converged"] == o["converged"]
    assert rel_err(x, o["x"]) <= 1e-10


@pytest.mark.parametrize("nlon,nlat,k,tiles,rows", [
    (2048, 320, 4, 0, 3),   # staged factors: 1-row bands; the SM count gives 3
    (4096, 40, 4, 0, 1),    # staged factors do not fit beside even one row
    (1024, 64, 3, 8, 8),    # 8-row bands asked for: too tall with staged factors
    (1000, 37, 5, 5, 8),    # ragged: nlon not a multiple of the register block, last band short
    (8192, 8, 4, 0, 1),     # the widest FP64 rows that fit
])
def test_fp64_global_factors_match_oracle(nlon, nlat, k, tiles, rows):
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=nlon + nlat)
    N = nlon * nlat
    faults = [(3, "r", N // 3, 62), (6, "ap", N // 2, 61)]
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, faults=faults)
    st, x, s = _solve(p, k, 1e-10, "fp64", faults, tiles=tiles)
    assert s["global_factors"] and -(-nlat // s["tiles"]) == rows, s
    assert s["steps"] == o["steps"] and s["detect_steps"] == o["detect_steps"] and s["converged"] == o["converged"]
    assert len(s["detect_steps"]) >= 1
    assert rel_err(x, o["x"]) <= 1e-10


def test_mixed_wide_rows_match_oracle():
    p = inputs.hill_problem(4096, 16, rhs="random", seed=32)
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-12)
    st, x, s = _solve(p, 4, 1e-10, "mixed")
    assert st == ftgcr.OK and s["converged"] and s["tiles"] == 16 and not s["split_rounds"]
    assert s["res_final_true"] <= 1e-10 * s["norm_R"]
    assert rel_err(x, o["x"]) <= 1e-7


def test_rows_too_wide_for_one_band_are_refused():
    # FP64 beyond about 8190 columns (factors from global memory); mixed beyond
    # about 8500 (split rounds)
    for (nlon, nlat), prec in (((12288, 4), "fp64"), ((16384, 4), "mixed")):
        p = inputs.hill_problem(nlon, nlat)
        with pytest.raises(ftgcr.FTGCRError) as ei:
            ftgcr.Solver(p.D, p.mu, precision=prec)
        assert ei.value.status == ftgcr.ERR_ARG


def test_fp64_batch_of_staged_and_global_factor_solves_equals_solo():
    # one launch holding both kinds runs the wide-row instance, which serves
    # both; each result is bitwise the one its handle gives alone
    probs = [inputs.hill_problem(n, m, rhs="random", seed=n + m) for n, m in ((1024, 64), (256, 128), (2000, 40))]
    tiles = [8, 0, 0]  # 8-row bands: global factors; 256 x 128: staged; 2000 x 40: 1-row bands, staged
    solvers = [ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="fp64", tiles=t) for p, t in zip(probs, tiles)]
    try:
        kinds = []
        R = [torch.from_numpy(p.R).cuda() for p in probs]
        alone, info_alone = [], []
        for s, r in zip(solvers, R):
            x = torch.zeros_like(r)
            s.solve(r, x, faults=[(4, "r", 77, 62)])
            alone.append(x.cpu().numpy())
            info_alone.append(s.stats())
            kinds.append(info_alone[-1]["global_factors"])
        assert kinds == [True, False, False], kinds
        xs = [torch.zeros_like(r) for r in R]
        ftgcr.solve_batch(solvers, R, xs, faults=[[(4, "r", 77, 62)]] * 3)
        torch.cuda.synchronize()
        for s, x, xa, ia in zip(solvers, xs, alone, info_alone):
            ib = s.stats()
            assert np.array_equal(x.cpu().numpy(), xa)
            assert ib["steps"] == ia["steps"] and ib["detect_steps"] == ia["detect_steps"]
    finally:
        for s in solvers:
            s.close()


def test_served_fp64_wide_rows_equal_solo():
    # the server's FP64 table launches the wide-row instance while a
    # global-factor request is in it, staged requests alongside
    probs = [inputs.hill_problem(n, m, rhs="random", seed=n * m) for n, m in ((4096, 24), (128, 64), (2048, 160))]
    with ftgcr.Server(max_slots=4, epoch_rounds=7) as srv:
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        xs = [torch.zeros_like(R) for R in Rs]
        tickets = [srv.submit(torch.from_numpy(p.D).cuda(), p.mu, R, x, k=4, tol=1e-10, precision="fp64")
                   for p, R, x in zip(probs, Rs, xs)]
        results = [srv.wait(t, timeout=120) for t in tickets]
    alone = []
    for p, (_, ss) in zip(probs, results):  # solo runs with the bands the server reported
        st, x, s = _solve(p, 4, 1e-10, "fp64", tiles=ss["tiles"])
        alone.append((x, s))
    assert [a[1]["global_factors"] for a in alone] == [True, False, True]
    for q, ((st, ss), (xa, sa)) in enumerate(zip(results, alone)):
        assert st == ftgcr.OK, (q, st)
        assert np.array_equal(xs[q].cpu().numpy(), xa), q
        assert ss["steps"] == sa["steps"] and ss["detect_steps"] == sa["detect_steps"]
