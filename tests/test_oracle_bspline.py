"""Pins for oracle/bspline.py (paper Appendix C): against scipy's B-splines and exact identities."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import Basis, clamped_uniform_knots, collocation, dstar, greville


@pytest.mark.parametrize("ny,p", [(9, 4), (17, 6), (33, 6), (20, 5)])
def test_matches_scipy_all_derivatives(ny, p):
    b = Basis(ny, p)
    for (t, order, pts, mats, nd) in ((b.t, p, b.g, b.Bg, 3), (b.t, p, b.gs, b.Bs, 4), (b.ts, p + 1, b.gs, b.Ss, 3)):
        n = len(t) - order
        for d in range(nd):
            ref = np.array([BSpline(t, np.eye(n)[j], order - 1)(pts, nu=d) for j in range(n)]).T
            scale = max(1.0, np.abs(ref).max())
            assert np.abs(ref - mats[d]).max() <= 1e-13 * scale, (order, d)


def test_dimensions_and_clamping():
    ny, p = 33, 6
    b = Basis(ny, p)
    assert b.Bg[0].shape == (ny, ny) and b.Ss[0].shape == (ny + 1, ny + 1)
    assert b.g[0] == -1.0 and b.g[-1] == 1.0 and b.gs[0] == -1.0 and b.gs[-1] == 1.0
    # clamped ends: value rows at the walls are unit vectors
    assert np.allclose(b.Bg[0][0], np.eye(ny)[0]) and np.allclose(b.Bg[0][-1], np.eye(ny)[-1])
    assert np.allclose(b.Ss[0][0], np.eye(ny + 1)[0]) and np.allclose(b.Ss[0][-1], np.eye(ny + 1)[-1])


def test_partition_of_unity_and_linear_precision():
    b = Basis(21, 6)
    x = np.linspace(-1, 1, 57)
    for t, order, g in ((b.t, 6, b.g), (b.ts, 7, b.gs)):
        M = collocation(t, order, x)
        assert np.abs(M.sum(1) - 1).max() < 1e-14
        # Greville abscissae reproduce x exactly (linear precision)
        assert np.abs(M @ g - x).max() < 1e-14


def test_polynomial_reproduction_and_derivative():
    """Degree <= p-1 polynomials are reproduced and differentiated exactly by the order-p space."""
    b = Basis(25, 6)
    poly = np.polynomial.Polynomial([0.3, -1.2, 0.7, 2.0, -0.5, 0.9])   # degree 5 = p - 1
    c = np.linalg.solve(b.Bg[0], poly(b.g))
    x = np.linspace(-1, 1, 41)
    for d in range(4):
        M = collocation(b.t, 6, x, d)
        ref = poly.deriv(d)(x)
        # rounding grows like (1/h)^d for the d-th derivative (h = knot spacing = 1/10 here)
        assert np.abs(M @ c - ref).max() < 1e-14 * np.abs(ref).max() * 20.0 ** (d + 1)


def test_integral_of_basis():
    """int B_j = (t_{j+k} - t_j) / k, with the oracle's own basis integrated by Gauss-Legendre per interval."""
    t = clamped_uniform_knots(6, 15)
    xg, wg = np.polynomial.legendre.leggauss(6)          # exact for degree <= 11
    brk = np.unique(t)
    pts, wts = [], []
    for a, b_ in zip(brk[:-1], brk[1:]):
        pts.append(0.5 * (b_ - a) * xg + 0.5 * (a + b_))
        wts.append(0.5 * (b_ - a) * wg)
    M = collocation(t, 6, np.concatenate(pts))
    integ = np.concatenate(wts) @ M
    assert np.abs(integ - (t[6:6 + 15] - t[:15]) / 6).max() < 1e-15


def test_dstar_is_exact_derivative():
    """d/dy of an order-(p+1) spline equals the order-p spline with coefficients D* c (Appendix C)."""
    b = Basis(29, 6)
    rng = np.random.default_rng(0)
    c = rng.normal(size=30)
    x = np.linspace(-1, 1, 97)
    lhs = collocation(b.ts, 7, x, 1) @ c
    rhs = collocation(b.t, 6, x, 0) @ (b.D @ c)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()
    assert np.count_nonzero(b.D) == 2 * 29   # bidiagonal


def test_greville_definition():
    t = clamped_uniform_knots(5, 11)
    g = greville(t, 5)
    assert np.allclose(g, [np.mean(t[j + 1:j + 5]) for j in range(11)])
    D = dstar(clamped_uniform_knots(6, 12), 6)
    assert D.shape == (11, 12)
