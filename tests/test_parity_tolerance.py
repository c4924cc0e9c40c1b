"""CPU checks of the tolerance the GPU parity tests use for dz/dt^{k_f} of a substage.

The bound (tests/_pairs.py, zdot_tolerance) comes from the 1/dt amplification of the BDF-like
guess (Eq. dzdt_guesses; Sec. 3.3.1 describes the resulting round-off floor of dz/dt). Two
properties make it a useful bound, and both are checked here on the oracle alone:
* the oracle's own response to a one-ulp-scale perturbation of its input state stays inside it;
* a real defect in dz/dt (one fixed-point application fewer, a wrong guess coefficient),
  planted in the oracle, lands far outside it.
"""
import numpy as np
import pytest

from _pairs import oracle_config, oracle_intermediates, rel, workload, zdot_tolerance
from oracle.lmvd import Substage
from paper_2206_09878_gb300.rt_inputs import WORKLOADS, rt_state

CASES = [{}, dict(nx=12, ny=11, nz=24, p=5, kmax=2)]


class WrongGuess(Substage):
    """Planted defect: the stage-' guess weighs z^{s-3} with 1.001 instead of 1 (Eq. dzdt_guesses)."""

    def bdf_guess(self):
        g = super().bdf_guess()
        if self.s % 2 == 1:
            g = g + 1e-3 * self.zh[2] / self.cfg.dt
        return g


def run(over, nsub=4, perturb=False, cls=Substage, **cfg_over):
    w = workload("rt32", **{k: v for k, v in over.items() if k in WORKLOADS["rt32"]})
    cfg = oracle_config(w, **{k: v for k, v in over.items() if k not in WORKLOADS["rt32"]}, **cfg_over)
    st = rt_state(**w)
    if perturb:
        rng = np.random.default_rng(7)
        for k in ("z", "om", "m2"):
            st[k] = st[k] * (1 + 2.0 ** -52 * rng.standard_normal(st[k].shape))
    S = cls(cfg)
    S.set_state(**st)
    out = []
    for _ in range(nsub):
        S.advance_substage()
        out.append(oracle_intermediates(S))
    return S, out


@pytest.mark.parametrize("over", CASES)
def test_one_ulp_input_noise_stays_inside(over):
    S, a = run(over)
    _, b = run(over, perturb=True)
    for s in range(len(a)):
        err = rel(b[s]["zdot"], a[s]["zdot"])
        assert err <= zdot_tolerance(S.cfg, a[s]), (s, err)


@pytest.mark.parametrize("over", CASES)
def test_planted_defects_in_dzdt_land_outside(over):
    S, a = run(over)
    # one fixed-point application fewer
    _, b = run(over, kf=S.cfg.kf - 1)
    # a guess coefficient off by 1e-3
    _, c = run(over, cls=WrongGuess)
    for bad in (b, c):
        ratio = max(rel(bad[s]["zdot"], a[s]["zdot"]) / zdot_tolerance(S.cfg, a[s]) for s in range(len(a)))
        assert ratio > 100.0, ratio


class SwappedMc(Substage):
    """Planted defect: m1^c and m3^c take each other's wavenumber factor (Eq. mc_recon: m1 = (k1/k) m_par,
    m3 = (k3/k) m_par, so swapping the factors swaps the two fields)."""

    def mc_from_rhot(self, rt):
        m1, m2, m3 = super().mc_from_rhot(rt)
        return m3, m2, m1


def test_downstream_bound_holds_for_rounding_and_fails_for_defect():
    """The bound on rho_t, m^c and the right-hand sides (NOISE_MARGIN x the rounding model's spread):
    another draw of the rounding model stays inside it; a planted defect in the m^c reconstruction
    lands far outside."""
    from _pairs import DOWNSTREAM, NOISE_MARGIN, PLAIN_TOL, downstream_floor, oracle_downstream, rounding_model
    w = workload("rt32")
    cfg = oracle_config(w)
    S = Substage(cfg)
    S.set_state(**rt_state(**w))
    for _ in range(3):
        S.advance_substage()
    zdot = S.trace["zdot"]
    ref, floor = downstream_floor(S, zdot)
    bound = {k: max(PLAIN_TOL, NOISE_MARGIN * floor[k]) for k in DOWNSTREAM}
    from _pairs import U64
    with rounding_model(S, U64, 99):
        other = oracle_downstream(S, zdot)
    for k in DOWNSTREAM:
        assert rel(other[k], ref[k]) <= bound[k], k
    B = SwappedMc(cfg)
    B.__dict__.update({k: v for k, v in S.__dict__.items()})
    bad = oracle_downstream(B, zdot)
    assert rel(bad["mc1"], ref["mc1"]) > 1e6 * bound["mc1"]


def test_rz_reference_from_a_given_state():
    """oracle_rz on the oracle's own state at the start of a substage reproduces that substage's R_z
    exactly, leaves the oracle untouched, and follows a change of the state (R_z is not a constant)."""
    from _pairs import oracle_rz
    w = workload("rt32")
    S = Substage(oracle_config(w))
    S.set_state(**rt_state(**w))
    S.advance_substage()
    before = {k: v.copy() for k, v in S.state().items()}
    S.advance_substage()
    z_after, rz_after, trace_keys = S.z.copy(), S.Rz, set(S.trace)
    rz = oracle_rz(S, before)
    assert np.array_equal(rz, S.Rz)
    assert np.array_equal(S.z, z_after) and S.Rz is rz_after and set(S.trace) == trace_keys
    moved = dict(before, z=before["z"] * (1 + 1e-6))
    assert rel(oracle_rz(S, moved), S.Rz) > 1e-9
