"""Pins of the oracle's per-mode y-systems by manufactured polynomial solutions.

The order-(p+1) space B* (Appendix C; p = 6, so piecewise degree 6) contains every polynomial of degree
<= 6, and interpolation at its Greville points reproduces such a polynomial exactly. So for a polynomial
P that satisfies a system's boundary rows, the system with right-hand side phi = P'' - k^2 P at its
collocation rows (zero in the boundary rows) must return P's own B* coefficients, found independently
by interpolation. Systems (A(k) = A2 - k^2 A0 + k A1):
* m^c (Sec. 4.2, Eq. COM_fourier + CF_fourier for m2^c), walls: P(+-1) = 0, collocation rows 1..ny-1;
* m2^d (Sec. 4.1, Eq. phi_poisson), walls: P(+-1) = P'(+-1) = 0, collocation rows 2..ny-2;
* the same with potential matching (Sec. 4.5, Eq. bc_both times k, Eq. md_bc): Robin rows
  k P(-1) - P'(-1) = 0 and k P(+1) + P'(+1) = 0; for m2^d also phi2(+-1) = P''(+-1) - k^2 P(+-1) = 0.
The polynomials satisfying the potential-matching rows are built from even and odd parts whose
coefficients solve those conditions in closed form (2 x 2 systems per part).
A dropped or mis-signed k-term, a wrong boundary row or a shifted collocation row fails these.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as Pl

from oracle.lmvd import Config, Operators

KS = (0.5, 1.0, 3.0, 10.0)


def _ops(bc):
    return Operators(Config(nx=8, ny=25, nz=8, bc=bc))


def _check(op, A2, A0, A1, k, coef, interior):
    """Solve A(k) x = phi with phi = P'' - k^2 P on the interior rows, compare with P's B* coefficients."""
    b = op.basis
    gs = b.gs
    n = len(gs)
    P = lambda y: Pl.polyval(y, coef)
    d2 = Pl.polyder(coef, 2)
    rhs = np.zeros(n)
    rhs[interior] = Pl.polyval(gs[interior], d2) - k * k * P(gs[interior])
    A = A2 - k * k * A0 + k * A1
    x = np.linalg.solve(A, rhs)
    expected = np.linalg.solve(np.asarray(b.Ss[0]), P(gs))
    assert np.abs(x - expected).max() <= 1e-10 * np.abs(expected).max(), (k, np.abs(x - expected).max())


def _robin_parts(k, phi_rows):
    """Even part 1 + a y^2 (+ b y^4) and odd part y + c y^3 (+ d y^5) satisfying k P(1) + P'(1) = 0 (and,
    with phi_rows, P''(1) - k^2 P(1) = 0); the conditions at y = -1 then hold by symmetry."""
    if not phi_rows:
        a = -k / (k + 2.0)                     # k (1 + a) + 2 a = 0
        c = -(1.0 + k) / (k + 3.0)             # k (1 + c) + 1 + 3 c = 0
        return np.array([1.0, 0.0, a]), np.array([0.0, 1.0, 0.0, c])
    # even: k (1 + a + b) + 2a + 4b = 0 ; 2a + 12b - k^2 (1 + a + b) = 0
    M = np.array([[k + 2.0, k + 4.0], [2.0 - k * k, 12.0 - k * k]])
    a, b = np.linalg.solve(M, np.array([-k, k * k]))
    # odd: k (1 + c + d) + 1 + 3c + 5d = 0 ; 6c + 20d - k^2 (1 + c + d) = 0
    M = np.array([[k + 3.0, k + 5.0], [6.0 - k * k, 20.0 - k * k]])
    c, d = np.linalg.solve(M, np.array([-(k + 1.0), k * k]))
    return np.array([1.0, 0.0, a, 0.0, b]), np.array([0.0, 1.0, 0.0, c, 0.0, d])


@pytest.mark.parametrize("k", KS)
def test_mc_system_walls(k):
    op = _ops("walls")
    ny = op.cfg.ny
    base = Pl.polymul([1.0, 0.0, -1.0], [0.3, -0.7, 1.1])          # (1 - y^2)(0.3 - 0.7 y + 1.1 y^2)
    _check(op, op.Amc2, op.Amc0, op.Amc1, k, base, np.arange(1, ny))


@pytest.mark.parametrize("k", KS)
def test_md_system_walls(k):
    op = _ops("walls")
    ny = op.cfg.ny
    base = Pl.polymul(Pl.polypow([1.0, 0.0, -1.0], 2), [0.4, 0.9])  # (1 - y^2)^2 (0.4 + 0.9 y)
    _check(op, op.Amd2, op.Amd0, op.Amd1, k, base, np.arange(2, ny - 1))


@pytest.mark.parametrize("k", KS)
def test_mc_system_potential(k):
    op = _ops("potential")
    ny = op.cfg.ny
    even, odd = _robin_parts(k, phi_rows=False)
    coef = Pl.polyadd(0.8 * even, -0.5 * odd)
    _check(op, op.Amc2, op.Amc0, op.Amc1, k, coef, np.arange(1, ny))


@pytest.mark.parametrize("k", KS)
def test_md_system_potential(k):
    op = _ops("potential")
    ny = op.cfg.ny
    even, odd = _robin_parts(k, phi_rows=True)
    coef = Pl.polyadd(0.6 * even, 1.3 * odd)
    # the conditions hold for the manufactured P itself (checked here, independently of the oracle)
    P = lambda y: Pl.polyval(y, coef)
    dP, d2P = Pl.polyder(coef), Pl.polyder(coef, 2)
    for y, s in ((-1.0, -1.0), (1.0, 1.0)):
        assert abs(k * P(y) + s * Pl.polyval(y, dP)) < 1e-12
        assert abs(Pl.polyval(y, d2P) - k * k * P(y)) < 1e-10 * max(1.0, k * k)
    _check(op, op.Amd2, op.Amd0, op.Amd1, k, coef, np.arange(2, ny - 1))


def test_wrong_k_sign_is_detected():
    """The pin is sensitive: the m2^d potential system with k replaced by -k in the Robin rows fails."""
    op = _ops("potential")
    ny = op.cfg.ny
    k = 1.0
    even, odd = _robin_parts(k, phi_rows=True)
    coef = Pl.polyadd(0.6 * even, 1.3 * odd)
    with pytest.raises(AssertionError):
        _check(op, op.Amd2, op.Amd0, -op.Amd1, k, coef, np.arange(2, ny - 1))
