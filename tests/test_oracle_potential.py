"""Pins for the potential-matching boundary conditions of oracle/lmvd.py (bc = "potential").

The paper's conditions (Sec. 4.5, Eq. bc_both, md_bc) make the truncated domain behave as the
unbounded one: outside [-1, 1] the momentum is the gradient of a decaying harmonic potential. So
for a source supported inside the domain, the truncated solves must reproduce the unbounded-line
solutions, which have closed forms:

* m^c (Sec. 4.2): psi'' - k^2 psi = -rho_t, m = grad psi, decaying at +-infinity:
  psi = (1/2k) int exp(-k|y-s|) rho_t(s) ds;
* m2^d (Eq. phi_poisson): m2'' - k^2 m2 = phi2, decaying: m2 = -(1/2k) int exp(-k|y-s|) phi2(s) ds.

For a Gaussian source exp(-s^2/sigma^2) the integral is, with c = sqrt(pi) sigma / 2 exp(k^2 sigma^2 / 4),
  I(y) = c [exp(-ky) erfc(k sigma/2 - y/sigma) + exp(ky) erfc(k sigma/2 + y/sigma)],
  I'(y) = c k [-exp(-ky) erfc(k sigma/2 - y/sigma) + exp(ky) erfc(k sigma/2 + y/sigma)].
No-slip walls give solutions that differ by tens of percent for k = 1, so these pins separate the
two boundary treatments and catch a sign error in either Robin row.

Two closed-form decay rates hold only with the potential-matching rows (constant density, KMM limit):
* phi2 = sin(pi (y+1)/2) (zero at both ends, Eq. md_bc) decays at mu (k^2 + pi^2/4);
* <m1> = cos(pi y) (zero slope at both ends: the Neumann rows on the plane means) decays at mu pi^2.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erfc

from oracle import banded
from oracle.lmvd import Config, Substage, _ax0


def green_integrals(y, k, sigma):
    c = np.sqrt(np.pi) * sigma / 2 * np.exp(k * k * sigma * sigma / 4)
    a = np.exp(-k * y) * erfc(k * sigma / 2 - y / sigma)
    b = np.exp(k * y) * erfc(k * sigma / 2 + y / sigma)
    return c * (a + b), c * k * (b - a)


def test_green_integral_closed_form_by_quadrature():
    """The erfc forms above against adaptive quadrature, split at the kink s = y."""
    k, sigma = 1.3, 0.2
    for y in (-0.9, -0.2, 0.0, 0.35, 1.0):
        I, dI = green_integrals(y, k, sigma)
        below = quad(lambda s: np.exp(-k * (y - s) - (s / sigma) ** 2), -np.inf, y, epsabs=1e-14)[0]
        above = quad(lambda s: np.exp(-k * (s - y) - (s / sigma) ** 2), y, np.inf, epsabs=1e-14)[0]
        assert abs(I - (below + above)) < 1e-12 and abs(dI - k * (above - below)) < 1e-12


def zero_state(S):
    cfg = S.cfg
    nxh = cfg.nx // 2 + 1
    z = np.zeros((cfg.ny, cfg.nz, nxh), complex)
    return dict(z=z, om=z.copy(), m2=np.zeros((cfg.ny + 1, cfg.nz, nxh), complex),
                mm1=np.zeros(cfg.ny), mm3=np.zeros(cfg.ny))


def interp_profile(S, f):
    return banded.solve(S.op.A_interp, f(S.op.basis.g).astype(complex))


MODES = [(0, 1), (0, 2), (1, 1), (7, 3)]     # (jz, kx) slots on an 8 x 8 grid: k = 1, 2, sqrt 2, sqrt 10


@pytest.mark.parametrize("bc", ["potential", "walls"])
def test_mc_matches_unbounded_solution(bc):
    """m^c from a Gaussian rho_t equals the unbounded-line solution only with potential matching."""
    cfg = Config(nx=8, ny=97, nz=8, bc=bc)
    S = Substage(cfg)
    op = S.op
    sigma = 0.2
    rt = np.zeros((cfg.ny, cfg.nz, cfg.nx // 2 + 1), complex)
    prof = interp_profile(S, lambda y: np.exp(-(y / sigma) ** 2))
    for jz, kx in MODES:
        rt[:, jz, kx] = prof
    m1, m2, m3 = S.mc_from_rhot(rt)
    gs, g = op.basis.gs, op.basis.g
    errs = []
    for jz, kx in MODES:
        k1, k3 = op.k1[jz, kx], op.k3[jz, kx]
        k = np.hypot(k1, k3)
        I_s, dI_s = green_integrals(gs, k, sigma)
        I_g, _ = green_integrals(g, k, sigma)
        m2_exact = dI_s / (2 * k)                       # m2 = psi'
        m1_exact = 1j * k1 * I_g / (2 * k)              # m1 = i k1 psi
        m3_exact = 1j * k3 * I_g / (2 * k)
        m2_num = (op.basis.Ss[0] @ m2[:, jz, kx])
        m1_num = op.basis.Bg[0] @ m1[:, jz, kx]
        m3_num = op.basis.Bg[0] @ m3[:, jz, kx]
        scale = np.abs(m2_exact).max()
        errs.append(max(np.abs(m2_num - m2_exact).max(), np.abs(m1_num - m1_exact).max(),
                        np.abs(m3_num - m3_exact).max()) / scale)
    assert np.all(np.isfinite(errs)) and len(errs) == len(MODES)
    if bc == "potential":
        assert max(errs) < 1e-6, errs
    else:
        assert min(errs) > 1e-2, errs


@pytest.mark.parametrize("bc", ["potential", "walls"])
def test_md_solve_matches_unbounded_solution(bc):
    """The m2^d system with phi2 = Gaussian at its interior rows and its four boundary rows."""
    cfg = Config(nx=8, ny=97, nz=8, bc=bc)
    S = Substage(cfg)
    op = S.op
    sigma = 0.2
    ny = cfg.ny
    rhs = np.zeros((ny + 1, cfg.nz, cfg.nx // 2 + 1), complex)
    gs = op.basis.gs
    for jz, kx in MODES:
        rhs[2:ny - 1, jz, kx] = np.exp(-(gs[2:ny - 1] / sigma) ** 2)
    m2 = op.solve_k2(op.Amd2, op.Amd0, rhs, op.Amd1)
    errs = []
    for jz, kx in MODES:
        k = np.sqrt(op.k2[jz, kx])
        I_s, _ = green_integrals(gs, k, sigma)
        exact = -I_s / (2 * k)
        num = op.basis.Ss[0] @ m2[:, jz, kx]
        errs.append(np.abs(num - exact).max() / np.abs(exact).max())
    assert np.all(np.isfinite(errs)) and len(errs) == len(MODES)
    if bc == "potential":
        assert max(errs) < 1e-6, errs
    else:
        assert min(errs) > 1e-2, errs


def const_density_cfg(**kw):
    c = dict(nx=4, ny=25, nz=4, rho_h=1.0, rho_l=1.0, re=1000.0, dt=1e-3, n_startup=2, bc="potential")
    c.update(kw)
    return Config(**c)


def test_phi2_dirichlet_mode_decay():
    """KMM limit: phi2 obeys d phi2/dt = mu (D^2 - k^2) phi2 with phi2(+-1) = 0 (Eq. md_bc)."""
    cfg = const_density_cfg(ny=33)
    S = Substage(cfg)
    op = S.op
    ny = cfg.ny
    st = zero_state(S)
    rhs = np.zeros((ny + 1, cfg.nz, cfg.nx // 2 + 1), complex)
    gs = op.basis.gs
    rhs[2:ny - 1, 0, 1] = 1e-8 * np.sin(np.pi * (gs[2:ny - 1] + 1) / 2)
    st["m2"] = op.solve_k2(op.Amd2, op.Amd0, rhs, op.Amd1)
    S.set_state(**st)
    a0 = S.m2[:, 0, 1].copy()
    nsteps = 50
    S.step(nsteps)
    rate = (1.0 + (np.pi / 2) ** 2) / cfg.re
    assert np.abs(S.m2[:, 0, 1] - a0 * np.exp(-rate * nsteps * cfg.dt)).max() < 1e-6 * np.abs(a0).max()


@pytest.mark.parametrize("bc", ["potential", "walls"])
def test_mean_neumann_decay(bc):
    """<m1> = cos(pi y) keeps its shape and decays at mu pi^2 only with the Neumann rows."""
    cfg = const_density_cfg(bc=bc)
    S = Substage(cfg)
    st = zero_state(S)
    st["mm1"] = np.real(interp_profile(S, lambda y: np.cos(np.pi * y)))
    S.set_state(**st)
    a0 = S.mm1.copy()
    nsteps = 50
    S.step(nsteps)
    err = np.abs(S.mm1 - a0 * np.exp(-np.pi ** 2 / cfg.re * nsteps * cfg.dt)).max() / np.abs(a0).max()
    if bc == "potential":
        assert err < 1e-6
    else:
        assert err > 1e-3


def rt_potential(seed=0):
    cfg = Config(nx=8, ny=17, nz=8, rho_l=1 / 3, re=200.0, dt=2e-3, n_startup=10, bc="potential",
                 y0=-2.0, y1=2.0, lx=1.0, lz=1.0)
    S = Substage(cfg)
    st = zero_state(S)
    rng = np.random.default_rng(seed)
    g = S.op.basis.g
    x = np.arange(8) / 8
    h = 0.05 * (np.cos(2 * np.pi * x)[None, :] + np.cos(2 * np.pi * x)[:, None])
    zf = 0.5 * (1 + np.tanh((g[:, None, None] - h[None]) / (2 * 0.05 * 4)))
    zh = np.fft.rfft2(zf, axes=(1, 2), norm="forward")
    zh[:, 4] = 0
    zh[:, :, 4] = 0
    st["z"] = banded.solve(S.op.A_interp, zh)
    gs = S.op.basis.gs
    for (jz, kx) in ((0, 1), (1, 1), (7, 2)):
        st["m2"][:, jz, kx] = 1e-3 * complex(rng.normal(), rng.normal()) * np.exp(-gs ** 2)
        st["om"][:, jz, kx] = 1e-3 * complex(rng.normal(), rng.normal()) * np.exp(-g ** 2)
    st["mm1"] = 1e-3 * np.real(interp_profile(S, lambda y: np.exp(-y ** 2)))
    return S, st


def test_boundary_rows_after_substages():
    """After each substage: Robin rows on m2^d and m2^c, phi2(+-1) = 0, Omega2(+-1) = 0, zero slope of
    the plane means and of z; and the m1, m3 lines of Eq. bc_both for m^d, which follow from them."""
    S, st = rt_potential()
    S.set_state(**st)
    op = S.op
    ny = S.cfg.ny
    Ss0, Ss1, Ss2 = op.basis.Ss[0], op.basis.Ss[1], op.basis.Ss[2]
    k = np.sqrt(op.k2)
    for _ in range(4):
        S.advance_substage()
        for m2 in (S.m2, S.trace["mc"][1]):
            scale = np.abs(m2).max()
            lo = k * _ax0(Ss0[:1], m2)[0] - _ax0(Ss1[:1], m2)[0]
            hi = k * _ax0(Ss0[ny:], m2)[0] + _ax0(Ss1[ny:], m2)[0]
            assert np.abs(lo * op.kmask).max() < 1e-12 * scale * ny ** 2
            assert np.abs(hi * op.kmask).max() < 1e-12 * scale * ny ** 2
        phi = _ax0(Ss2, S.m2) - op.k2 * _ax0(Ss0, S.m2)
        assert np.abs(phi[[0, ny]] * op.kmask).max() < 1e-12 * np.abs(phi).max()
        assert np.abs(S.om[[0, ny - 1]]).max() < 1e-14 * np.abs(S.om).max()
        for f in (S.mm1, S.mm3):
            assert np.abs(op.basis.Bg[1][[0, ny - 1]] @ f).max() < 1e-12 * max(np.abs(f).max(), 1e-300) * ny
        dz = _ax0(op.basis.Bg[1][[0, ny - 1]], S.z)
        assert np.abs(dz).max() < 1e-12 * np.abs(S.z).max() * ny
        # Eq. bc_both, second and third lines, for m^d: m1 = -+ i k1/k m2 at y = +-1
        m1, m3 = S.md_components(S.m2, S.om, S.mm1, S.mm3)
        safe = np.where(op.kmask, k, 1.0)
        for row, b, sgn in ((0, 0, 1.0), (ny - 1, ny, -1.0)):
            m2b = S.m2[b]
            assert np.abs((m1[row] - sgn * 1j * op.k1 / safe * m2b) * op.kmask).max() < 1e-10 * np.abs(S.m2).max()
            assert np.abs((m3[row] - sgn * 1j * op.k3 / safe * m2b) * op.kmask).max() < 1e-10 * np.abs(S.m2).max()


def test_potential_mass_and_hermitian():
    S, st = rt_potential(seed=3)
    S.set_state(**st)
    for _ in range(3):
        S.advance_substage()
        res = S.mass_residual(S.trace["rho_t"], S.trace["mc"])
        assert np.abs(res).max() < 1e-13 * max(1e-30, np.abs(S.trace["rho_t"]).max())
        col = S.z[:, :, 0]
        nz = S.cfg.nz
        for jz in range(1, nz // 2):
            assert np.abs(col[:, jz] - np.conj(col[:, nz - jz])).max() < 1e-15 * max(1, np.abs(col).max())
