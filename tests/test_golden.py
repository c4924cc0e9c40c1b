"""Pins against values the paper prints (fixtures under tests/golden/, each citing its passage):
* the constants of the scalar test system of Sec. 3.3.1 are the ones the oracle's stepper test uses;
* the paper's case table (Table RT_casedetails) and its domains are the ones the input module carries,
  and the paper set-ups built from them (rtp32, rtp128, rtp128_hi) take Re, domain and time step from it.
"""
import inspect
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_e1_constants_are_the_papers():
    from oracle import ode_e1
    g = {r[0]: complex(float(r[1]), float(r[2])) for r in _rows("e1_test_problem.txt")}
    assert (ode_e1.C1, ode_e1.C2, ode_e1.C3, ode_e1.C4) == (g["c1"], g["c2"], g["c3"], g["c4"])
    defaults = {k: v.default for k, v in inspect.signature(ode_e1.run).parameters.items()}
    assert defaults["z0"] == g["z0"] and defaults["md0"] == g["md0"]
    assert defaults["kf"] == g["kf"].real and defaults["beta_p"] == g["beta_p"].real
    assert defaults["beta_n"] == g["beta_n"].real


def test_case_table_is_the_papers():
    from paper_2206_09878_gb300.rt_inputs import PAPER_CASES, PAPER_DOMAINS
    rows = _rows("rt_case_table.txt")
    cases = [r for r in rows if r[0] != "domain"]
    assert len(cases) == len(PAPER_CASES)
    for dim, at, re, dom, dts in cases:
        row = PAPER_CASES[(int(dim), float(at))]
        assert row["re"] == float(re) and row["dt_scaled"] == float(dts)
        # the last 3D row prints V^{2D,2}; as a 3D case the module reads it as V^{3D,2}
        expect = "3D,2" if (dim, at, dom) == ("3", "0.925", "2D,2") else dom
        assert row["domain"] == expect
    for _, name, y0, y1, mesh in (r for r in rows if r[0] == "domain"):
        d = PAPER_DOMAINS[name]
        assert (d[0], d[1]) == (float(y0), float(y1))
        assert d[2] == tuple(int(v) for v in mesh.split("x"))


@pytest.mark.parametrize("name", ["rtp32", "rtp128", "rtp128_hi"])
def test_paper_setups_follow_the_table(name):
    from paper_2206_09878_gb300.rt_inputs import PAPER_CASES, PAPER_DOMAINS, PAPER_RT, paper_rt_config
    w = PAPER_RT[name]
    row = PAPER_CASES[(3, w["at"])]
    y0, y1, mesh = PAPER_DOMAINS[row["domain"]]
    assert (w["y0"], w["y1"]) == (y0, y1)
    if name != "rtp32":                                # rtp32: a small mesh on the same domain
        assert (w["nx"], w["ny"], w["nz"]) == mesh
    c = paper_rt_config(**w)
    assert c["re"] == row["re"]
    assert c["dt"] * np.sqrt(w["at"]) == pytest.approx(row["dt_scaled"], rel=1e-15)
    assert c["rho_l"] == pytest.approx((1 - w["at"]) / (1 + w["at"]))
