"""Pins of the oracle's preconditioner: P is the within-row (zonal) part of L
plus the diagonal of the rest, and solve_P inverts it (checked against dense
LAPACK solves and the residual P(P^-1 r) - r)."""
import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import inputs


def _dense(p, fn):
    return oracle.dense_matrix(fn, p.nlat, p.nlon)


@pytest.mark.parametrize("nlon,nlat", [(8, 4), (12, 5), (3, 2)])
def test_P_is_row_block_of_L(nlon, nlat):
    p = inputs.hill_problem(nlon, nlat, h0=0.3, width=0.7, centre=(2.0, -0.3))
    L = _dense(p, lambda v: oracle.apply_L(p.D, p.mu, v))
    P = _dense(p, lambda v: oracle.apply_P(p.D, p.mu, v))
    for a in range(p.nlat * p.nlon):
        for b in range(p.nlat * p.nlon):
            if a // nlon == b // nlon:
                assert P[a, b] == pytest.approx(L[a, b], rel=1e-14, abs=0)
            else:
                assert P[a, b] == 0.0
    # the rest of L is exactly the meridional coupling: zero diagonal
    assert np.all(np.diag(L - P) == pytest.approx(0.0, abs=1e-13 * np.abs(np.diag(L)).max()))


@pytest.mark.parametrize("kind", [oracle.PRECOND_LINE, oracle.PRECOND_JACOBI, oracle.PRECOND_IDENTITY])
@pytest.mark.parametrize("nlon,nlat", [(8, 4), (16, 8), (5, 3), (3, 1)])
def test_solve_P_matches_dense_solve(kind, nlon, nlat):
    p = inputs.hill_problem(nlon, nlat, h0=0.2)
    r = inputs.uniform_pm1(7, (nlat, nlon))
    e = oracle.solve_P(p.D, p.mu, r, kind)
    if kind == oracle.PRECOND_LINE:
        P = _dense(p, lambda v: oracle.apply_P(p.D, p.mu, v))
    elif kind == oracle.PRECOND_JACOBI:
        L = _dense(p, lambda v: oracle.apply_L(p.D, p.mu, v))
        P = np.diag(np.diag(L))
    else:
        P = np.eye(nlat * nlon)
    ref = np.linalg.solve(P, r.ravel()).reshape(nlat, nlon)
    np.testing.assert_allclose(e, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nlon,nlat", [(256, 128), (1024, 512), (100, 37)])
def test_line_solve_residual_on_anisotropic_rows(nlon, nlat):
    # near the poles Tx / (mu A) ~ 1/cos^2(theta): nearly singular rows
    p = inputs.hill_problem(nlon, nlat)
    r = inputs.uniform_pm1(3, (nlat, nlon))
    e = oracle.solve_P(p.D, p.mu, r)
    back = oracle.apply_P(p.D, p.mu, e)
    rel = np.abs(back - r).max(axis=1) / np.abs(r).max(axis=1)
    assert rel.max() < 1e-9, rel.max()


def test_line_preconditioner_is_exact_for_single_row():
    # nlat = 1: L has no meridional coupling, so P = L and e = L^-1 r
    p = inputs.hill_problem(16, 1)
    r = inputs.uniform_pm1(5, (1, 16))
    e = oracle.solve_P(p.D, p.mu, r)
    np.testing.assert_allclose(oracle.apply_L(p.D, p.mu, e), r, rtol=1e-12, atol=1e-14)


def test_preconditioner_sign_matches_L():
    # e = P^-1 r has the sign convention of L^-1: <r, L e> > 0 for r != 0
    p = inputs.hill_problem(32, 16)
    r = inputs.uniform_pm1(9, (16, 32))
    e = oracle.solve_P(p.D, p.mu, r)
    assert oracle.dot(r, oracle.apply_L(p.D, p.mu, e)) > 0
