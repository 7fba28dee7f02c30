"""Pins of the oracle's fault-tolerance semantics (Algorithm 1, red part;
Section 2 and Section 3): invariants that hold exactly whatever the operator.

* x and p never enter beta, alpha or r, so flips there are passive: the norm
  sequence is bitwise that of the fault-free run and nothing is detected,
  and the solution differs from the fault-free one at the flipped entry only
  (every recurrence of x and p is entrywise).
* A flip that sets bit 62 of an r entry with |v| < 2 multiplies it by 2^1024
  (Inf or a huge value): always detected in the step it fires.
* A fault detected in the step it fires, that did not reach the backup,
  replays the same cycle from the backup: the solution is bitwise the
  fault-free one and at most k + 1 steps are spent (the failed step plus a
  cycle, Section 2 "at most a full iteration").
* A flip of L(p) that overflows <L(p), L(p)> makes beta = 0, r unchanged,
  so the norm test sees equality and flags it (">=" reading)."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import inputs


def test_flip_bit_is_xor_of_ieee_pattern():
    g = inputs.SplitMix64(5)
    for _ in range(200):
        v = 2.0 * g.uniform() - 1.0
        b = g.below(64)
        ref = (np.array([v]).view(np.uint64) ^ np.uint64(1 << b)).view(np.float64)[0]
        got = oracle.flip_bit(v, b)
        assert np.array([got]).view(np.uint64)[0] == np.array([ref]).view(np.uint64)[0]


@pytest.fixture(scope="module")
def base():
    p = inputs.hill_problem(64, 32, rhs="random", seed=1)
    ff = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    return p, ff


@pytest.mark.parametrize("vec", ["x", "p"])
def test_flips_in_x_and_p_are_passive(base, vec):
    p, ff = base
    N = p.nlat * p.nlon
    for trial in range(12):
        f = inputs.sweep_flip(100, trial, ff["steps"], N, vecs=(vec,))
        o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[f])
        assert o["faults_detected"] == 0 and o["faults_injected"] == 1
        assert np.array_equal(o["nrm2_hist"], ff["nrm2_hist"])


def _entry(vec_hist_fn, p, ff, step):
    return None


def test_bit62_flip_of_small_r_entry_is_detected_and_replayed(base):
    p, ff = base
    N = p.nlat * p.nlon
    k = 4
    for step in range(2, ff["steps"]):
        # index with |r| < 2 at that step: the residual entries are O(1) or smaller
        idx = (step * 7919) % N
        f = (step, "r", idx, 62)
        o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, faults=[f])
        assert o["detect_steps"] == [step], (step, o["detect_steps"])
        assert np.array_equal(o["x"], ff["x"])
        assert 1 <= o["steps"] - ff["steps"] <= k + 1


def test_overflowing_Lp_flip_gives_beta_zero_and_is_detected(base):
    p, ff = base
    N = p.nlat * p.nlon
    for step in (3, 6, 9):
        f = (step, "ap", (step * 131) % N, 62)
        o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[f])
        assert step in o["detect_steps"]
        assert o["converged"]


def test_small_e_flips_go_undetected_and_converge(base):
    # low mantissa bits of e: consistent p and L(p), norm keeps decreasing
    p, ff = base
    N = p.nlat * p.nlon
    for trial in range(8):
        g = inputs.SplitMix64(300 + trial)
        f = (1 + g.below(ff["steps"] - 1), "e", g.below(N), g.below(20))
        o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[f])
        assert o["faults_detected"] == 0 and o["converged"]
        assert o["res_true"] <= 2e-10 * np.sqrt(o["nrm2_R"])


def test_fault_after_convergence_never_fires(base):
    p, ff = base
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[(ff["steps"] + 5, "r", 3, 62)])
    assert o["faults_injected"] == 0 and np.array_equal(o["x"], ff["x"])


def test_first_step_fault_restores_clean_initial_backup(base):
    # the backup starts as the initial state, before the first step's flips
    p, ff = base
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[(1, "r", 17, 62)])
    assert o["detect_steps"] == [1]
    assert np.array_equal(o["x"], ff["x"]) and o["steps"] == ff["steps"] + 1


def test_wasted_steps_bounded_by_cycle(base):
    p, ff = base
    N = p.nlat * p.nlon
    k = 4
    for trial in range(40):
        f = inputs.sweep_flip(7, trial, ff["steps"], N, vecs=("r", "ap"))
        o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, faults=[f])
        assert o["converged"]
        if o["faults_detected"]:
            # each detection costs at most the failed step and one cycle
            assert len(o["detect_steps"]) == 1


def test_nan_in_residual_is_a_fault(base):
    p, ff = base
    # exponent of a value in [1, 2) becomes all ones -> NaN (mantissa != 0) or Inf
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[(4, "r", 5, 62), (4, "r", 5, 61)])
    assert 4 in o["detect_steps"]


@pytest.mark.parametrize("vec,bit", [("x", 40), ("p", 40), ("p", 57), ("x", 62), ("p", 61)])
def test_passive_flips_stay_in_their_entry(base, vec, bit):
    p, ff = base
    N = p.nlon * p.nlat
    for step, idx in ((2, 17), (7, N // 2 + 3), (ff["steps"], N - 5)):
        o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10, faults=[(step, vec, idx, bit)])
        assert o["faults_injected"] == 1 and o["faults_detected"] == 0
        x, x0 = o["x"].ravel(), ff["x"].ravel()
        other = np.ones(N, dtype=bool)
        other[idx] = False
        assert np.array_equal(x[other], x0[other]), (vec, bit, step, idx)
        assert not np.array_equal(x[idx], x0[idx])
