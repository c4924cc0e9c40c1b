"""Pin for the stepper logic (Algorithm 1, Eq. dzdt_guesses, Eq. y_k): the paper's scalar test system.

Sec. 3.3.1: with k_f = 4, beta' = -4, beta^n = 0, z and m^d converge at second order to the
reference obtained by integrating dz/dt = M2 / (1 - M1) directly.
"""
import math

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
