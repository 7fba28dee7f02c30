"""Pins of the oracle's grid geometry and operator (Eq. (1)) against facts the
mathematics fixes: the sphere's area, symmetry and definiteness of the
finite-volume matrix, exact conservation, and second-order consistency with
the continuous operator div(D grad phi) on the sphere."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_07210_gb300 import inputs


@pytest.mark.parametrize("nlon,nlat", [(8, 4), (64, 32), (40, 21), (3, 1)])
def test_total_area_is_4pi(nlon, nlat):
    _, _, area = oracle.geometry(nlon, nlat)
    assert abs(nlon * area.sum() - 4 * math.pi) < 1e-12


def test_area_is_band_area():
    # exact zonal band areas: 2 pi (sin b - sin a) / nlon per cell
    nlon, nlat = 12, 6
    _, _, area = oracle.geometry(nlon, nlat)
    edges = np.linspace(-math.pi / 2, math.pi / 2, nlat + 1)
    exact = 2 * math.pi * (np.sin(edges[1:]) - np.sin(edges[:-1])) / nlon
    np.testing.assert_allclose(area, exact, rtol=1e-13)


@pytest.mark.parametrize("nlon,nlat", [(8, 4), (16, 8), (12, 7)])
def test_operator_symmetric_and_definite(nlon, nlat):
    p = inputs.hill_problem(nlon, nlat, h0=0.3, width=0.6, centre=(1.0, 0.4))
    L = oracle.dense_matrix(lambda v: oracle.apply_L(p.D, p.mu, v), nlat, nlon)
    assert np.array_equal(L, L.T), "finite-volume matrix must be exactly symmetric"
    np.linalg.cholesky(-L)  # -L positive definite
    _, _, area = oracle.geometry(nlon, nlat)
    lam_min = np.linalg.eigvalsh(-L).min()
    # -L = (flux part, positive semi-definite) + mu diag(A)
    assert lam_min >= p.mu * area.min() * (1 - 1e-12)


def test_flux_part_annihilates_constants():
    nlon, nlat = 16, 8
    p = inputs.hill_problem(nlon, nlat)
    _, _, area = oracle.geometry(nlon, nlat)
    out = oracle.apply_L(p.D, p.mu, np.ones((nlat, nlon)))
    np.testing.assert_array_equal(out, -(p.mu * area)[:, None] * np.ones((nlat, nlon)))
    out0 = oracle.apply_L(p.D, 0.0, np.full((nlat, nlon), 3.5))
    assert np.abs(out0).max() == 0.0


def test_operator_sparsity_pattern():
    # 5-point stencil, periodic in longitude, no coupling across the poles
    nlon, nlat = 8, 4
    p = inputs.hill_problem(nlon, nlat)
    L = oracle.dense_matrix(lambda v: oracle.apply_L(p.D, p.mu, v), nlat, nlon)
    for a in range(nlat * nlon):
        ja, ia = divmod(a, nlon)
        for b in range(nlat * nlon):
            jb, ib = divmod(b, nlon)
            neigh = (ja == jb and (ib - ia) % nlon in (0, 1, nlon - 1)) or (ia == ib and abs(ja - jb) == 1)
            if not neigh:
                assert L[a, b] == 0.0
            else:
                assert L[a, b] != 0.0


def _sphere_divgrad(D_expr, phi_expr):
    """Exact div(D grad phi) on the unit sphere (sympy), lambda = longitude,
    theta = latitude."""
    sp = pytest.importorskip("sympy")
    lam, th = sp.symbols("lam th", real=True)
    D = D_expr(sp, lam, th)
    phi = phi_expr(sp, lam, th)
    expr = (sp.diff(D * sp.diff(phi, lam) / sp.cos(th), lam) + sp.diff(sp.cos(th) * D * sp.diff(phi, th), th)) / sp.cos(th)
    f_D = sp.lambdify((lam, th), D, "numpy")
    f_phi = sp.lambdify((lam, th), phi, "numpy")
    f_L = sp.lambdify((lam, th), expr, "numpy")
    return f_D, f_phi, f_L


def _consistency_error(nlon, nlat, fD, fphi, fL, lat_max):
    lam, th = inputs.cell_centres(nlon, nlat)
    LAM, TH = np.meshgrid(lam, th)
    D = np.broadcast_to(fD(LAM, TH), LAM.shape).astype(float).copy()
    phi = np.broadcast_to(fphi(LAM, TH), LAM.shape).astype(float).copy()
    _, _, area = oracle.geometry(nlon, nlat)
    Lphi = oracle.apply_L(D, 0.0, phi) / area[:, None]
    exact = fL(LAM, TH)
    band = np.abs(th) < lat_max
    return np.abs(Lphi - exact)[band].max()


@pytest.mark.parametrize(
    "case",
    [
        # Laplacian eigenfunctions: -l(l+1) Y
        (lambda sp, l, t: sp.Integer(1), lambda sp, l, t: sp.sin(t)),
        (lambda sp, l, t: sp.Integer(1), lambda sp, l, t: sp.sin(t) * sp.cos(t) * sp.cos(l)),
        # variable coefficient in latitude and longitude
        (lambda sp, l, t: 1 + sp.sin(t) / 2, lambda sp, l, t: sp.sin(t)),
        (lambda sp, l, t: 1 + sp.cos(t) * sp.cos(l) / 3, lambda sp, l, t: sp.cos(t) * sp.sin(2 * l)),
        (lambda sp, l, t: 1 - sp.Rational(1, 10) * sp.exp(-((l - 3) ** 2 + t ** 2) * 4),
         lambda sp, l, t: sp.cos(t) ** 2 * sp.cos(l) + sp.sin(t)),
    ],
)
def test_second_order_consistency(case):
    fD, fphi, fL = _sphere_divgrad(*case)
    errs = [_consistency_error(16 * 2 ** q, 8 * 2 ** q, fD, fphi, fL, math.radians(60)) for q in range(4)]
    rates = [errs[q] / errs[q + 1] for q in range(3)]
    assert errs[-1] < 1e-2, errs
    # O(h^2): mean rate over three refinements near 4, every single rate well
    # above the 2 of a first-order (e.g. wrong-metric) discretisation
    assert (errs[0] / errs[-1]) ** (1 / 3) > 3.4, (errs, rates)
    assert min(rates) > 2.8, (errs, rates)


def test_eigenvalue_of_Y1():
    # D = 1, mu = 0, Y = sin(theta): div grad Y = -2 Y, exactly second order
    nlon, nlat = 256, 128
    lam, th = inputs.cell_centres(nlon, nlat)
    Y = np.tile(np.sin(th)[:, None], (1, nlon))
    _, _, area = oracle.geometry(nlon, nlat)
    LY = oracle.apply_L(np.ones_like(Y), 0.0, Y) / area[:, None]
    assert np.abs(LY + 2 * Y).max() < 1e-3


def test_flow_rhs_is_conservative():
    p = inputs.hill_problem(64, 32)
    assert abs(p.R.sum()) < 1e-14 * np.abs(p.R).sum() * 10
    np.testing.assert_allclose(p.R.sum(axis=1), 0.0, atol=1e-15)


def test_flow_rhs_is_divergence_of_ambient_flow():
    # R = div(D v_a) with v_a = (cos theta, 0): the potential phi = 0 with D = 1
    # gives zero divergence (solid-body rotation is divergence free)
    D = np.ones((16, 32))
    assert np.abs(inputs.flow_rhs(D)).max() < 1e-15
