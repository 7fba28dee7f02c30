"""Pins of the oracle's FT-GCR(k) iteration (Algorithm 1) in fault-free runs:
the exact discrete solution (dense LAPACK), manufactured solutions, the
minimisation property (strictly decreasing residual norms, Section 2), the
one-step convergence with an exact preconditioner (fixes the sign of beta),
finite termination, and orthogonality of L(p^l) within a cycle."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import inputs


def _dense_L(p):
    return oracle.dense_matrix(lambda v: oracle.apply_L(p.D, p.mu, v), p.nlat, p.nlon)


@pytest.mark.parametrize("nlon,nlat,k", [(16, 8, 4), (32, 16, 3), (12, 7, 5), (8, 1, 2)])
@pytest.mark.parametrize("precond", [oracle.PRECOND_LINE, oracle.PRECOND_JACOBI, oracle.PRECOND_IDENTITY])
def test_matches_dense_solve(nlon, nlat, k, precond):
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=11, h0=0.2)
    L = _dense_L(p)
    xs = np.linalg.solve(L, p.R.ravel()).reshape(p.R.shape)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-12, precond=precond)
    assert o["converged"]
    cond = np.linalg.cond(L)
    err = np.linalg.norm(o["x"] - xs) / np.linalg.norm(xs)
    assert err <= 10 * cond * 1e-12, (err, cond)
    assert o["res_true"] <= 1.01e-12 * np.sqrt(o["nrm2_R"]) + 1e-15


@pytest.mark.parametrize("nlon,nlat", [(64, 32), (48, 20)])
def test_manufactured_solution(nlon, nlat):
    p = inputs.hill_problem(nlon, nlat)
    phi = inputs.uniform_pm1(21, (nlat, nlon))
    R = oracle.apply_L(p.D, p.mu, phi)
    o = oracle.ftgcr(p.D, R, p.mu, 4, 1e-13)
    assert o["converged"]
    assert np.abs(o["x"] - phi).max() < 1e-9


@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("precond", [oracle.PRECOND_LINE, oracle.PRECOND_JACOBI, oracle.PRECOND_IDENTITY])
def test_norms_strictly_decrease_without_faults(k, precond):
    p = inputs.hill_problem(64, 32, rhs="random", seed=3)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-10, precond=precond)
    assert o["converged"] and o["faults_detected"] == 0
    h = np.concatenate([[o["nrm2_0"]], o["nrm2_hist"]])
    assert np.all(np.diff(h) < 0)
    assert np.all(o["events"][:-1] == oracle.EVENT_ACCEPT) and o["events"][-1] == oracle.EVENT_EXIT


def test_exact_preconditioner_converges_in_one_step():
    # P = L: e = L^-1 r, so L(p^0) = r^0 and beta = -1 makes r^1 = 0.  The
    # printed sign of beta would double the residual instead.
    p = inputs.hill_problem(8, 4, rhs="random", seed=5)
    Linv = np.linalg.inv(_dense_L(p))
    o = oracle.ftgcr(p.D, p.R, p.mu, 3, 1e-10, precond=oracle.PRECOND_DENSE, dense_pinv=Linv)
    assert o["converged"] and o["steps"] == 1
    assert o["beta_hist"][0] == pytest.approx(-1.0, abs=1e-12)


def test_finite_termination_when_k_covers_the_space():
    # without restarts GCR terminates in at most N steps (exact arithmetic)
    p = inputs.hill_problem(4, 3, rhs="random", seed=8)
    N = p.nlat * p.nlon
    o = oracle.ftgcr(p.D, p.R, p.mu, N, 1e-11, precond=oracle.PRECOND_IDENTITY)
    assert o["converged"] and o["steps"] <= N + 1


def test_orthogonality_and_norm_identity_within_cycles():
    k = 5
    p = inputs.hill_problem(16, 8, rhs="random", seed=4)
    o = oracle.ftgcr(p.D, p.R, p.mu, k, 1e-12, trace_lp=True, precond=oracle.PRECOND_JACOBI)
    lp = o["lp_trace"].reshape(o["steps"], -1)
    n = o["steps"]
    for c0 in range(0, n, k):
        blk = lp[c0:min(c0 + k, n)]
        G = blk @ blk.T
        d = np.sqrt(np.diag(G))
        C = G / np.outer(d, d)
        off = np.abs(C - np.eye(len(blk))).max()
        assert off < 1e-8, (c0, off)
    # ||r^{nu+1}||^2 = ||r^nu||^2 - beta^2 ||L p^nu||^2  (minimisation along L p)
    h = np.concatenate([[o["nrm2_0"]], o["nrm2_hist"]])
    pred = h[:-1] - o["beta_hist"] ** 2 * np.einsum("ij,ij->i", lp, lp)
    np.testing.assert_allclose(h[1:], pred, rtol=1e-7, atol=1e-12 * h[0])


def test_recurrence_residual_tracks_true_residual():
    p = inputs.hill_problem(128, 64)
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    assert o["converged"]
    assert abs(np.sqrt(o["nrm2_final"]) - o["res_true"]) <= 1e-9 * np.sqrt(o["nrm2_R"])


def test_zero_rhs_and_exact_guess():
    p = inputs.hill_problem(16, 8, rhs="random", seed=2)
    o = oracle.ftgcr(p.D, np.zeros_like(p.R), p.mu, 4, 1e-10, x0=np.ones_like(p.R))
    assert o["converged"] and o["steps"] == 0 and np.all(o["x"] == 0)
    phi = inputs.uniform_pm1(3, p.R.shape)
    R = oracle.apply_L(p.D, p.mu, phi)
    o = oracle.ftgcr(p.D, R, p.mu, 4, 1e-10, x0=phi)
    assert o["converged"] and o["steps"] == 0 and np.array_equal(o["x"], phi)


def test_step_limit():
    p = inputs.hill_problem(64, 32, rhs="random", seed=2)
    o = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-14, max_steps=7)
    assert not o["converged"] and o["steps"] == 7 and o["status"] == 1
