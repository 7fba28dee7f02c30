"""Oracle pins for the paper's data-loss fault model, the unprotected GCR(k)
mode and the singular mu = 0 (pure Neumann Poisson) problem.

- SplitMix64, the counter-based generator both sides use for the flips of a
  data-loss event, reproduces the reference outputs published with the
  generator (seed 1234567).
- A data-loss event (Section 3: a number of entries of e inside one process
  block each suffer one bit flip) equals, bitwise, the plan of single e flips
  that an independent Python restatement of the event computes.
- Unprotected GCR(k) (the paper's baseline, Section 3) is FT-GCR(k) without the
  fault test: identical when nothing goes wrong, never restores otherwise.
- mu = 0: with a consistent right-hand side (zero sum) the oracle converges to
  the minimum-norm solution up to a constant, as a dense least-squares solve
  says."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import inputs

# Reference outputs of SplitMix64 for seed 1234567 (the test vector published
# with the generator's reference implementation).
SM64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                16408922859458223821]


def test_splitmix64_reproduces_the_published_reference_outputs():
    assert [oracle.splitmix64(1234567, i) for i in range(1, 6)] == SM64_1234567
    assert [int(v) for v in inputs.splitmix64(1234567, 5)] == SM64_1234567


def _event_flips(N, rank, nranks, count, seed, nbits):
    """Independent restatement of a data-loss event's flips."""
    b0, b1 = rank * N // nranks, (rank + 1) * N // nranks
    z = inputs.splitmix64(seed, count).astype(object)
    return [(b0 + int(v) % (b1 - b0), (int(v) >> 32) % nbits) for v in z]


@pytest.mark.parametrize("count,rank,nranks,step", [(1, 0, 1, 3), (7, 2, 5, 2), (300, 4, 8, 5), (40, 0, 3, 1)])
def test_data_loss_event_equals_its_single_flips(count, rank, nranks, step):
    p = inputs.hill_problem(32, 16, rhs="random", seed=5)
    N = p.R.size
    seed = 0xC0FFEE + count
    ev = (step, rank, nranks, count, seed, 64)
    a = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, losses=[ev])
    flips = [(step, "e", idx, bit) for idx, bit in _event_flips(N, rank, nranks, count, seed, 64)]
    b = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=flips)
    assert a["loss_events"] == 1
    assert np.array_equal(a["x"], b["x"])
    assert a["steps"] == b["steps"] and a["detect_steps"] == b["detect_steps"]
    assert np.array_equal(a["nrm2_hist"], b["nrm2_hist"], equal_nan=True)


def test_data_loss_flips_stay_inside_the_rank_block():
    N = 32 * 16
    for rank, nranks in [(0, 7), (3, 7), (6, 7)]:
        b0, b1 = rank * N // nranks, (rank + 1) * N // nranks
        fl = _event_flips(N, rank, nranks, 500, 99, 32)
        assert all(b0 <= i < b1 for i, _ in fl) and all(0 <= b < 32 for _, b in fl)
        assert len({i for i, _ in fl}) > 0.6 * min(500, b1 - b0)  # spread over the block


def test_a_repeated_event_cancels_itself():
    p = inputs.hill_problem(32, 16, rhs="random", seed=6)
    ev = (3, 1, 4, 50, 1234, 64)
    clean = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    twice = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, losses=[ev, ev])  # XOR twice at the same step
    assert twice["loss_events"] == 2
    assert np.array_equal(clean["x"], twice["x"]) and clean["steps"] == twice["steps"]


def test_events_at_steps_never_reached_do_not_fire():
    p = inputs.hill_problem(32, 16, rhs="random", seed=6)
    clean = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    late = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, losses=[(clean["steps"] + 5, 0, 1, 10, 7, 64)])
    assert late["loss_events"] == 0 and np.array_equal(clean["x"], late["x"])


def test_unprotected_equals_protected_without_faults():
    for k in (1, 3, 5):
        p = inputs.hill_problem(64, 32, rhs="random", seed=k)
        a = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10)
        b = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, protect=False)
        assert np.array_equal(a["x"], b["x"]) and a["steps"] == b["steps"]
        assert np.array_equal(a["nrm2_hist"], b["nrm2_hist"], equal_nan=True)


def test_unprotected_gcr_never_restores():
    p = inputs.hill_problem(64, 32, rhs="random", seed=8)
    N = p.R.size
    base = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    # bit 62 of a small r entry: the entry becomes huge, ||r|| jumps at step 6
    r_small = [(6, "r", i, 62) for i in range(0, N, N // 3)]
    prot = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=r_small)
    unprot = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=r_small, protect=False, max_steps=base["steps"] + 200)
    assert prot["faults_detected"] >= 1 and prot["restarts"] >= 1
    assert unprot["faults_detected"] == 0 and unprot["restarts"] == 0
    h = unprot["nrm2_hist"]
    assert not (h[5] < h[4])  # the norm did grow at the faulty step and nothing reacted
    assert unprot["steps"] > prot["steps"] or not unprot["converged"]


def test_mu_zero_consistent_problem_matches_least_squares():
    nlon, nlat = 12, 6
    p = inputs.hill_problem(nlon, nlat, rhs="flow", mu_hat=0.0)
    assert p.mu == 0.0
    R = p.R - p.R.mean()  # exactly consistent: zero sum
    o = oracle.ftgcr(p.D, R, 0.0, 6, 1e-12)
    assert o["converged"]
    L = oracle.dense_matrix(lambda v: oracle.apply_L(p.D, 0.0, v), nlat, nlon)
    assert np.allclose(L.sum(axis=1), 0.0, atol=1e-12)  # constants span the null space
    xs = np.linalg.lstsq(L, R.ravel(), rcond=None)[0]
    x = o["x"].ravel()
    d = (x - x.mean()) - (xs - xs.mean())
    assert np.linalg.norm(d) <= 1e-8 * np.linalg.norm(xs)
    assert np.linalg.norm(L @ x - R.ravel()) <= 1e-12 * np.linalg.norm(R) * 10
