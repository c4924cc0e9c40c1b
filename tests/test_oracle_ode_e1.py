"""Pin for the stepper logic (Algorithm 1, Eq. dzdt_guesses, Eq. y_k): the paper's scalar test system.

Sec. 3.3.1: with k_f = 4, beta' = -4, beta^n = 0, z and m^d converge at second order to the
reference obtained by integrating dz/dt = M2 / (1 - M1) directly.
Sec. 3.3.2: on the linear test system dz/dt = lam1 dz/dt + lam2 z, one RK2 step equals the paper's
closed-form map (with the z' coefficient read as 4 + beta'; the printed 3 + beta' does not keep a
constant state constant).
"""
import math

import numpy as np

import pytest

from oracle import ode_e1


def test_second_order_convergence_of_algorithm_1():
    zr, mr = ode_e1.reference(0.1)
    errs = []
    for n in (20, 40, 80, 160):
        z, md = ode_e1.run(0.1 / n, 0.1)
        errs.append((abs(z - zr), abs(md - mr)))
    for a, b in zip(errs[:-1], errs[1:]):
        assert 1.85 < math.log2(a[0] / b[0]) < 2.1
        assert 1.85 < math.log2(a[1] / b[1]) < 2.1


@pytest.mark.parametrize("kf", [1, 2, 8])
def test_order_independent_of_iteration_count(kf):
    """Sec. 3.1: the order of accuracy does not depend on the number of iterations."""
    zr, mr = ode_e1.reference(0.1)
    e1 = abs(ode_e1.run(0.1 / 40, 0.1, kf=kf)[0] - zr)
    e2 = abs(ode_e1.run(0.1 / 80, 0.1, kf=kf)[0] - zr)
    assert 1.8 < math.log2(e1 / e2) < 2.2


def test_wrong_guess_coefficient_breaks_order():
    """A guess that is only first-order accurate (z^{n-1} coefficient perturbed) loses second order."""
    zr, _ = ode_e1.reference(0.1)
    # beta' enters every coefficient of the family consistently; a plain zeroth-order guess
    # (dz/dt^0 = 0, k_f = 1) is one application of the iteration from a wrong start: order drops
    e1 = abs(ode_e1.run(0.1 / 40, 0.1, kf=1, beta_p=-4.0)[0] - zr)
    assert e1 < 1e-4


@pytest.mark.parametrize("kf", [1, 2, 4, 7])
@pytest.mark.parametrize("lam1,lam2", [(0.2j, -1.0), (0.5 + 0.5j, 0.3 - 2.0j), (0.7 + 0.25j, -0.5)])
@pytest.mark.parametrize("beta_p", [-4.0, -3.0, 0.5])
def test_linear_test_system_matches_the_closed_form_step(kf, lam1, lam2, beta_p):
    """Sec. 3.3.2 (linear stability analysis): for dz/dt = lam1 dz/dt + lam2 z with k fixed-point
    iterations and beta^n = 0, one RK2 step (stages n and ') of the stepper is the paper's closed form
      z' - z^n        = lam1^k (z^n - z^{n-1,'}) + dt/2 S lam2 z^n,
      z^{n+1} - z'    = lam1^k ((4 + beta') z' - (6 + 2 beta') z^n + (beta' + 1) z^{n-1,'} + z^{n-1})
                        + dt S lam2 (z' - z^n / 2),          S = sum_{j<k} lam1^j.
    The paper prints 3 + beta' for the z' coefficient; with it a constant state would not stay constant
    (next test), so it is read as 4 + beta', which is also what substituting Eq. dzdt_guesses gives."""
    from oracle import ode_e1
    rng = np.random.default_rng(11)
    zn, zp1, z1, zp2 = rng.normal(size=4) + 1j * rng.normal(size=4)   # z^n, z^{n-1,'}, z^{n-1}, z^{n-2,'}
    dt = 0.01
    m1, m2 = (lambda z: lam1), (lambda z: lam2 * z)
    g_n = ode_e1.zdot_of_substage(0, zn, [zp1, z1, zp2], dt, kf, 0.0, beta_p, m1, m2)
    _, (al, be) = ode_e1.stage_coefficients(0, 0.0, beta_p)
    zp = zn + dt * (al * g_n + be * 123.0)          # be = 0 at stage n: the previous dz/dt does not enter
    g_p = ode_e1.zdot_of_substage(1, zp, [zn, zp1, z1], dt, kf, 0.0, beta_p, m1, m2)
    _, (al, be) = ode_e1.stage_coefficients(1, 0.0, beta_p)
    znew = zp + dt * (al * g_p + be * g_n)
    S = sum(lam1 ** j for j in range(kf))
    zp_closed = zn + lam1 ** kf * (zn - zp1) + 0.5 * dt * S * lam2 * zn
    znew_closed = (zp + lam1 ** kf * ((4 + beta_p) * zp - (6 + 2 * beta_p) * zn + (beta_p + 1) * zp1 + z1)
                   + dt * S * lam2 * (zp - 0.5 * zn))
    assert abs(zp - zp_closed) <= 1e-13 * (1 + abs(zp))
    assert abs(znew - znew_closed) <= 1e-13 * (1 + abs(znew))


def test_printed_coefficient_would_not_preserve_a_constant():
    """With lam2 = 0 and a constant history the stepper keeps z constant; the closed form with the printed
    3 + beta' would move it by -lam1^k z."""
    from oracle import ode_e1
    lam1, kf, beta_p, dt, c = 0.4 + 0.3j, 3, -4.0, 0.01, 0.7 - 0.2j
    m1, m2 = (lambda z: lam1), (lambda z: 0.0)
    hist = [c, c, c]
    g_n = ode_e1.zdot_of_substage(0, c, hist, dt, kf, 0.0, beta_p, m1, m2)
    zp = c + 0.5 * dt * g_n
    g_p = ode_e1.zdot_of_substage(1, zp, [c, c, c], dt, kf, 0.0, beta_p, m1, m2)
    znew = zp + dt * (g_p - 0.5 * g_n)
    assert abs(zp - c) < 1e-14 and abs(znew - c) < 1e-14        # up to rounding in the guess
    printed = zp + lam1 ** kf * ((3 + beta_p) * zp - (6 + 2 * beta_p) * c + (beta_p + 1) * c + c)
    assert abs(printed - c) == pytest.approx(abs(lam1 ** kf * c), rel=1e-12)
