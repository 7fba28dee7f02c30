"""Streamed step rounds (FTGCR_FLAG_STREAMED_ROUNDS): every CTA walks one
tall band row by row, its operand rows staged into shared memory by
per-thread asynchronous copies, and the band's edge rows take their stencil in
a second pass.  Forced here on grids the oracle solves in seconds: one-row to
64-row bands (the tallest allowed), more bands than SMs, rows of one, two and
a ragged second chunk of columns,
k = 1..8, flips of every vector, data-loss events, and batches that mix
streamed solves with solves of the other layouts.  Every solution matches the
FP64 oracle to 1e-10 at tol 1e-13; batched results equal solo results
bitwise."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs
from tests import sweep_worker
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13
# (nlon, nlat, k, rhs, tiles): tiles 0 = one band per SM
CASES = [
    (1024, 64, 4, "flow", 0),      # 64 one-row bands: every stencil in the second pass
    (1024, 512, 4, "flow", 0),     # 152 bands of 3-4 rows
    (1024, 512, 8, "random", 0),
    (2048, 300, 2, "flow", 0),     # two chunks per row
    (2044, 300, 3, "flow", 40),    # a short second chunk, padded line-solve pieces; 7-8-row bands
    (1000, 33, 1, "random", 2),    # one short chunk; two tall bands
    (1024, 33, 5, "random", 1),    # one band: every row interior
    (2048, 64, 4, "flow", 64),     # two chunks per row, one-row bands
    (1024, 128, 4, "flow", 2),     # 64-row bands, the tallest a streamed band may be
    (1024, 130, 3, "flow", 2),     # 65-row bands asked for: raised to three bands of 43-44 rows
    (1024, 512, 4, "random", 256), # 2-row bands, more bands than SMs: a CTA walks two a round
]


@pytest.fixture(scope="module")
def oracle_x():
    import oracle

    oracle.build()
    args = [(n, m, k, TOL, rhs, 5, None) for n, m, k, rhs, _ in CASES]
    with mp.get_context("spawn").Pool(min(8, len(args))) as pool:
        res = pool.map(sweep_worker.oracle_solution, args)
    return dict(zip([c[:4] for c in CASES], res))


def _solve(p, k, tiles, faults=(), rounds="streamed", tol=TOL, losses=()):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision="mixed", tiles=tiles, rounds=rounds) as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st = s.solve(R, x, faults=faults, losses=losses) if losses else s.solve(R, x, faults=faults)
        return st, x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}_k{c[2]}_{c[3]}_t{c[4]}" for c in CASES])
def test_streamed_matches_oracle(oracle_x, case):
    nlon, nlat, k, rhs, tiles = case
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=5)
    st, x, info = _solve(p, k, tiles)
    assert st == ftgcr.OK and info["converged"], info
    assert info["streamed_rounds"], info
    assert info["res_final_true"] <= TOL * info["norm_R"]
    xref, conv, _ = oracle_x[case[:4]]
    assert conv
    assert rel_err(x, xref) <= 1e-10


def test_streamed_bands_stay_within_64_rows():
    """A tiling whose bands would pass 64 rows is raised to the fewest bands
    of at most 64 rows (at 1024 x 9729, one band more than there are SMs);
    a tiling of 64-row bands is kept.  The 10 M-point solve is checked by its
    own true residual."""
    for nlat, tiles, want in ((130, 2, 3), (128, 2, 2), (9729, 0, 153)):
        p = inputs.hill_problem(1024, nlat)
        st, x, info = _solve(p, 4, tiles, tol=1e-10)
        assert info["tiles"] == want and info["streamed_rounds"], (nlat, tiles, info["tiles"])
        assert st == ftgcr.OK and info["converged"]
        assert info["res_final_true"] <= 1e-10 * info["norm_R"]


def test_streamed_is_deterministic_and_close_to_fused():
    p = inputs.hill_problem(1024, 128, rhs="random", seed=9)
    st1, x1, i1 = _solve(p, 4, 0)
    st2, x2, i2 = _solve(p, 4, 0)
    assert np.array_equal(x1, x2) and i1["steps"] == i2["steps"]
    st3, x3, i3 = _solve(p, 4, 0, rounds="fused")
    assert not i3["streamed_rounds"]
    assert rel_err(x1, x3) <= 1e-10


@pytest.mark.parametrize("vec", ["x", "r", "p", "ap", "e"])
def test_streamed_with_flips_converges_to_oracle(oracle_x, vec):
    nlon, nlat, k, rhs, tiles = CASES[1]
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=5)
    N = nlon * nlat
    xref = oracle_x[CASES[1][:4]][0]
    det = 0
    for trial in range(4):
        f = inputs.sweep_flip(300 + trial, trial, 12, N, nbits=32, vecs=(vec,))
        st, x, info = _solve(p, k, tiles, faults=[f])
        assert st == ftgcr.OK and info["converged"], (f, info)
        assert info["faults_injected"] == 1, (f, info)
        assert rel_err(x, xref) <= 1e-10, f
        det += info["faults_detected"]
    # a flip of the sign or exponent of an r or L(p) entry is detected
    if vec in ("r", "ap"):
        f = (3, inputs.VEC_CODES[vec], N // 2 + 17, 30)
        st, x, info = _solve(p, k, tiles, faults=[f])
        assert info["faults_detected"] >= 1 and info["converged"]
        assert rel_err(x, xref) <= 1e-10


def test_streamed_with_data_loss_converges():
    nlon, nlat, k, rhs, tiles = CASES[1]
    p = inputs.hill_problem(nlon, nlat, rhs=rhs, seed=5)
    losses = [(4, 3, 72, 50, 1234), (7, 40, 72, 2000, 99)]
    st, x, info = _solve(p, k, tiles, losses=losses)
    assert st == ftgcr.OK and info["converged"] and info["loss_events"] == 2, info
    with ftgcr.Solver(p.D, p.mu, k=k, tol=TOL, precision="mixed", rounds="fused") as s:
        R = torch.from_numpy(p.R).cuda()
        xf = torch.zeros_like(R)
        s.solve(R, xf)
    assert rel_err(x, xf.cpu().numpy()) <= 1e-10


def test_batch_mixing_streamed_and_other_layouts_is_bitwise_solo():
    shapes = [(1024, 128, "streamed", 4), (256, 128, "auto", 4), (1024, 64, "streamed", 8), (4096, 24, "split", 4),
              (128, 64, "fused", 2), (2048, 40, "streamed", 3)]
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(70 + q)) for q, (n, m, _, _) in enumerate(shapes)]
    solvers = [ftgcr.Solver(p.D, p.mu, k=k, tol=1e-10, precision="mixed", rounds=r)
               for p, (_, _, r, k) in zip(probs, shapes)]
    try:
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        faults = [()] * len(probs)
        faults[0] = [(3, 1, 5000, 30)]
        faults[2] = [(2, 4, 777, 28)]
        alone = []
        for s, R, f in zip(solvers, Rs, faults):
            x = torch.zeros_like(R)
            s.solve(R, x, faults=f)
            alone.append((x.clone(), s.stats()))
        xs = [torch.zeros_like(R) for R in Rs]
        ftgcr.solve_batch(solvers, Rs, xs, faults=faults)
        torch.cuda.synchronize()
        for q, (s, x) in enumerate(zip(solvers, xs)):
            st = s.stats()
            assert torch.equal(x, alone[q][0]), q
            for key in ("steps", "detect_steps", "outer", "converged", "res_final_true"):
                assert st[key] == alone[q][1][key], (q, key)
        assert alone[0][1]["streamed_rounds"] and alone[3][1]["split_rounds"]
    finally:
        for s in solvers:
            s.close()


def test_server_mixing_streamed_and_other_layouts_is_bitwise_solo():
    """Served requests in every layout, streamed among them (the launch then runs the
    streamed instance for all), host arrays, each result bitwise the solo one."""
    shapes = [(1024, 96, "streamed"), (256, 128, "auto"), (2048, 40, "streamed"), (4096, 24, "split"),
              (128, 64, "fused"), (1024, 64, "streamed")]
    probs = [inputs.hill_problem(n, m, **inputs.random_hill(90 + q)) for q, (n, m, _) in enumerate(shapes)]
    alone = []
    for p, (_, _, r) in zip(probs, shapes):
        with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision="mixed", rounds=r) as s:
            x = np.zeros_like(p.R)
            s.solve(p.R, x)
            alone.append((x, s.stats()))
    with ftgcr.Server(max_slots=4, epoch_rounds=7) as srv:
        xs = [np.zeros_like(p.R) for p in probs]
        ts = [srv.submit(torch.from_numpy(p.D).cuda(), p.mu, p.R, x, precision="mixed", rounds=r, coeff_key=q + 1)
              for q, (p, x, (_, _, r)) in enumerate(zip(probs, xs, shapes))]
        res = [srv.wait(t, timeout=120) for t in ts]
    for q, (st, ss) in enumerate(res):
        assert st == ftgcr.OK, q
        assert np.array_equal(xs[q], alone[q][0]), q
        assert ss["steps"] == alone[q][1]["steps"] and ss["streamed_rounds"] == alone[q][1]["streamed_rounds"]


def test_streamed_flag_rejected_where_it_cannot_run():
    # nlon not a multiple of 4; per-lane chunks of 40 (not a power of two);
    # chunks of 8 (rows under 993 columns)
    for nlon in (1022, 1028, 256):
        p = inputs.hill_problem(nlon, 8)
        with pytest.raises(ftgcr.FTGCRError):
            ftgcr.Solver(p.D, p.mu, precision="mixed", rounds="streamed")
    q = inputs.hill_problem(1024, 8)
    with pytest.raises(ftgcr.FTGCRError):
        ftgcr.Solver(q.D, q.mu, precision="fp64", rounds="streamed")
