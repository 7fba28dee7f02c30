"""Serving (ftgcr_server_*): independent requests of mixed sizes and both
precisions, submitted while others run, each come back bitwise equal (solution
and counters) to the same request solved alone; handles are reused across
requests of the same shape with new coefficients; admission respects the
memory budget; invalid requests are refused at submit; host inputs holding
non-finite values complete with an argument error.  Each solo run uses the
row bands the server reported for the request."""
import time

import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("steps", "cycles", "restarts", "faults_injected", "faults_detected", "outer", "converged", "detect_steps",
        "res_final_rec", "res_final_true", "status")


def _requests(seed):
    """(problem, precision, faults, oracle_order) of a small mix; shapes repeat
    with new hills so that pooled handles get new coefficients, and some FP64
    requests of a shape ask for the oracle's operation order (a handle of
    their own: pooled handles match on the flags too)."""
    shapes = [(128, 64), (64, 32), (256, 128), (128, 64), (40, 21), (512, 256), (256, 128), (64, 32), (1024, 512),
              (128, 64), (100, 7), (256, 128)]
    out = []
    for q, (nlon, nlat) in enumerate(shapes):
        p = inputs.hill_problem(nlon, nlat, **inputs.random_hill(seed + q))
        prec = "mixed" if q % 3 == 1 else "fp64"
        nb = 32 if prec == "mixed" else 64
        faults = ()
        if q == 2:
            faults = [(3, "r", 100, nb - 2)]
        if q == 5:
            faults = [(5, "ap", 777, nb - 2), (9, "e", 12345, 20)]
        if q == 7:
            faults = [(4, "r", 33, nb - 2)]
        out.append((p, prec, faults, prec == "fp64" and q in (3, 9, 10)))
    return out


def _alone(p, prec, faults, k, tiles=0, oracle_order=False):
    # tiles: the bands the server reported for the request
    with ftgcr.Solver(p.D, p.mu, k=k, tol=1e-10, precision=prec, tiles=tiles, oracle_order=oracle_order) as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        s.solve(R, x, faults=faults)
        return x.cpu().numpy(), s.stats()


@pytest.mark.parametrize("epoch_rounds", [5, 48])
def test_served_results_are_bitwise_the_solo_results(epoch_rounds):
    reqs = _requests(101)
    k = 4
    with ftgcr.Server(max_slots=4, epoch_rounds=epoch_rounds) as srv:
        Ds = [torch.from_numpy(p.D).cuda() for p, _, _, _ in reqs]
        Rs = [torch.from_numpy(p.R).cuda() for p, _, _, _ in reqs]
        xs = [torch.zeros_like(R) for R in Rs]
        tickets = []
        for q, (p, prec, f, oo) in enumerate(reqs):
            tickets.append(srv.submit(Ds[q], p.mu, Rs[q], xs[q], k=k, tol=1e-10, precision=prec, faults=f,
                                      oracle_order=oo))
            if q % 4 == 3:
                time.sleep(0.002)  # later requests arrive while earlier ones run
        if epoch_rounds == 5:  # completion queue
            got = {}
            for _ in tickets:
                nx = srv.next(timeout=120)
                assert nx is not None
                got[nx[0]] = (nx[1], nx[2])
            results = [got.get(t) for t in tickets]
        else:
            results = [srv.wait(t, timeout=120) for t in tickets]
        info = srv.info()
    assert info["completed"] == len(reqs) and info["queued"] == 0 and info["running"] == 0
    for q, res in enumerate(results):
        assert res is not None, q
        st, ss = res
        p, prec, f, oo = reqs[q]
        xa, sa = _alone(p, prec, f, k, ss["tiles"], oo)
        assert st == ftgcr.OK and sa["converged"], (q, st, sa)
        assert np.array_equal(xs[q].cpu().numpy(), xa), q
        for key in KEYS:
            assert ss[key] == sa[key], (q, key, ss[key], sa[key])


def test_host_arrays_are_served_like_device_arrays():
    p = inputs.hill_problem(128, 64, **inputs.random_hill(7))
    with ftgcr.Server(max_slots=2) as srv:
        x = np.zeros_like(p.R)
        t = srv.submit(p.D, p.mu, p.R, x, k=4, precision="mixed")
        st, ss = srv.wait(t, timeout=60)
    xa, sa = _alone(p, "mixed", (), 4, ss["tiles"])
    assert st == ftgcr.OK
    assert np.array_equal(x, xa)
    assert ss["steps"] == sa["steps"]


def test_a_pooled_handle_takes_the_next_requests_coefficients():
    a = inputs.hill_problem(256, 128, **inputs.random_hill(3))
    b = inputs.hill_problem(256, 128, **inputs.random_hill(4))
    assert not np.array_equal(a.D, b.D) and a.mu == b.mu
    with ftgcr.Server(max_slots=2) as srv:
        out = []
        for p in (a, b, a):
            x = torch.zeros(p.R.shape, dtype=torch.float64, device="cuda")
            st, ss = srv.wait(srv.submit(torch.from_numpy(p.D).cuda(), p.mu, torch.from_numpy(p.R).cuda(), x),
                              timeout=60)
            assert st == ftgcr.OK
            out.append((x.cpu().numpy(), ss))
        assert srv.info()["handles"] == 1
    for p, (x, ss) in zip((a, b, a), out):
        xa, sa = _alone(p, "fp64", (), 4, ss["tiles"])
        assert np.array_equal(x, xa) and ss["steps"] == sa["steps"]


def test_coefficient_keys_reuse_set_up_handles_correctly():
    a = inputs.hill_problem(256, 128, **inputs.random_hill(13))
    b = inputs.hill_problem(256, 128, **inputs.random_hill(14))
    Da, Db = torch.from_numpy(a.D).cuda(), torch.from_numpy(b.D).cuda()
    with ftgcr.Server(max_slots=2) as srv:
        out = []
        for p, D, key in ((a, Da, 1), (b, Db, 2), (a, Da, 1), (b, Db, 2), (a, Da, 0)):
            x = torch.zeros(p.R.shape, dtype=torch.float64, device="cuda")
            st, ss = srv.wait(srv.submit(D, p.mu, torch.from_numpy(p.R).cuda(), x, coeff_key=key), timeout=60)
            assert st == ftgcr.OK
            out.append((p, x.cpu().numpy(), ss))
    for p, x, ss in out:
        xa, sa = _alone(p, "fp64", (), 4, ss["tiles"])
        assert np.array_equal(x, xa) and ss["steps"] == sa["steps"]


def test_admission_stays_within_the_budget():
    small = ftgcr.footprint(256, 128, 4)
    budget = int(small * 2.5)
    with ftgcr.Server(budget_bytes=budget, max_slots=8, epoch_rounds=16) as srv:
        big = inputs.hill_problem(1024, 512)
        with pytest.raises(ftgcr.FTGCRError) as ei:
            srv.submit(big.D, big.mu, big.R, np.zeros_like(big.R))
        assert ei.value.status == ftgcr.ERR_BUDGET
        probs = [inputs.hill_problem(256, 128, **inputs.random_hill(50 + q)) for q in range(5)]
        Rs = [torch.from_numpy(p.R).cuda() for p in probs]
        xs = [torch.zeros_like(R) for R in Rs]
        ts = [srv.submit(torch.from_numpy(p.D).cuda(), p.mu, R, x) for p, R, x in zip(probs, Rs, xs)]
        peak = 0
        while True:
            i = srv.info()
            peak = max(peak, i["bytes_in_use"])
            if i["completed"] == len(ts):
                break
            time.sleep(0.0005)
        res = [srv.wait(t, timeout=60) for t in ts]
    assert peak <= budget
    assert all(r[0] == ftgcr.OK for r in res)
    for p, x, (st, ss) in zip(probs, xs, res):
        xa, sa = _alone(p, "fp64", (), 4, ss["tiles"])
        assert np.array_equal(x.cpu().numpy(), xa) and ss["steps"] == sa["steps"]


def test_invalid_requests_are_refused_at_submit():
    p = inputs.hill_problem(64, 32)
    with ftgcr.Server(max_slots=2) as srv:
        with pytest.raises(ftgcr.FTGCRError) as ei:
            srv.submit(p.D, p.mu, p.R, np.zeros_like(p.R), faults=[(1, "r", p.R.size, 3)])  # index out of range
        assert ei.value.status == ftgcr.ERR_ARG
        with pytest.raises(ftgcr.FTGCRError):
            srv.submit(p.D, p.mu, p.R, np.zeros_like(p.R), k=0)
        with pytest.raises(ftgcr.FTGCRError):
            srv.poll(12345)


def test_non_finite_host_inputs_complete_with_an_argument_error():
    # host arrays are staged and checked on the device: the request does not
    # start, completes with ERR_ARG and leaves x as it was; the others run
    p = inputs.hill_problem(64, 32)
    with ftgcr.Server(max_slots=2) as srv:
        bad = p.R.copy()
        bad[3, 5] = np.nan
        x_bad = np.full_like(p.R, 0.25)
        t_bad = srv.submit(p.D, p.mu, bad, x_bad)
        x_inf = np.zeros_like(p.R)
        x_inf[1, 1] = -np.inf
        t_inf = srv.submit(p.D, p.mu, p.R, x_inf, precision="mixed")
        x_ok = np.zeros_like(p.R)
        t_ok = srv.submit(p.D, p.mu, p.R, x_ok)
        st_bad, _ = srv.wait(t_bad, timeout=60)
        st_inf, _ = srv.wait(t_inf, timeout=60)
        st_ok, ss = srv.wait(t_ok, timeout=60)
    assert st_bad == ftgcr.ERR_ARG and np.all(x_bad == 0.25)
    assert st_inf == ftgcr.ERR_ARG
    xa, sa = _alone(p, "fp64", (), 4, ss["tiles"])
    assert st_ok == ftgcr.OK and np.array_equal(x_ok, xa) and ss["steps"] == sa["steps"]


def test_max_points_limits_the_running_solves_and_keeps_results():
    """With a limit of one 256x128 grid per table, at most one mixed solve
    runs at a time (a larger request runs alone), FP64 solves are limited
    separately, and every result is still the solo result."""
    shapes = [(256, 128, "mixed"), (256, 128, "mixed"), (512, 256, "mixed"), (256, 128, "fp64"), (256, 128, "mixed"),
              (128, 64, "fp64"), (256, 128, "mixed")]
    probs = [(inputs.hill_problem(n, m, **inputs.random_hill(300 + q)), prec) for q, (n, m, prec) in enumerate(shapes)]
    with ftgcr.Server(max_slots=8, epoch_rounds=6) as srv:
        srv.set_max_points(256 * 128)
        Rs = [torch.from_numpy(p.R).cuda() for p, _ in probs]
        xs = [torch.zeros_like(R) for R in Rs]
        ts = [srv.submit(torch.from_numpy(p.D).cuda(), p.mu, R, x, precision=prec)
              for (p, prec), R, x in zip(probs, Rs, xs)]
        peak = 0
        while srv.info()["completed"] < len(ts):
            peak = max(peak, srv.info()["running"])
            time.sleep(0.0002)
        res = [srv.wait(t, timeout=60) for t in ts]
    assert peak <= 2  # one per precision table
    assert all(r[0] == ftgcr.OK for r in res)
    for (p, prec), x, (st, ss) in zip(probs, xs, res):
        xa, sa = _alone(p, prec, (), 4, ss["tiles"])
        assert np.array_equal(x.cpu().numpy(), xa) and ss["steps"] == sa["steps"]
    with ftgcr.Server() as srv:
        with pytest.raises(ftgcr.FTGCRError):
            srv.set_max_points(-1)


def test_requests_whose_handles_are_prepared_beside_a_running_launch_match_solo():
    """Requests of one shape with eight different coefficient keys, submitted
    while a long solve runs: handles are created or rebuilt beside the
    running launch, and every result is the solo result."""
    big = inputs.hill_problem(1024, 512, **inputs.random_hill(400))
    probs = [inputs.hill_problem(256, 128, **inputs.random_hill(410 + q)) for q in range(8)]
    with ftgcr.Server(max_slots=16, epoch_rounds=4) as srv:
        Rb = torch.from_numpy(big.R).cuda()
        xb = torch.zeros_like(Rb)
        tb = srv.submit(torch.from_numpy(big.D).cuda(), big.mu, Rb, xb, precision="mixed", coeff_key=1)
        Ds = [torch.from_numpy(p.D).cuda() for p in probs]
        Rs = [torch.from_numpy(p.R).pin_memory() for p in probs]
        xs = [torch.zeros(p.R.shape, dtype=torch.float64).pin_memory() for p in probs]
        ts = [srv.submit(D, p.mu, R, x, precision="mixed", coeff_key=10 + q)
              for q, (p, D, R, x) in enumerate(zip(probs, Ds, Rs, xs))]
        # the same keys again: pooled handles already set up from them
        xs2 = [torch.zeros(p.R.shape, dtype=torch.float64).pin_memory() for p in probs]
        ts2 = [srv.submit(D, p.mu, R, x, precision="mixed", coeff_key=10 + q)
               for q, (p, D, R, x) in enumerate(zip(probs, Ds, Rs, xs2))]
        res = [srv.wait(t, timeout=60) for t in ts + ts2]
        rb = srv.wait(tb, timeout=60)
    assert rb[0] == ftgcr.OK and all(r[0] == ftgcr.OK for r in res)
    xa, _ = _alone(big, "mixed", (), 4, rb[1]["tiles"])
    assert np.array_equal(xb.cpu().numpy(), xa)
    for q, p in enumerate(probs):
        xa, sa = _alone(p, "mixed", (), 4, res[q][1]["tiles"])
        assert np.array_equal(xs[q].numpy(), xa) and np.array_equal(xs2[q].numpy(), xa)
