"""Closed-form pins of the oracle's convective right-hand side, R_z, f'(z) and the L tail.

The states here are chosen so that the continuous equations have an exact answer that can be
written down without the method:

* a passive scalar carried by a uniform stream at constant density (Sec. 2.1, Eq. zeqn_imp with
  f' = 0): dz/dt = -(U d/dx + W d/dz) z + kappa lap z, exactly, for a single Fourier mode;
* an Omega2 mode and a phi2 mode carried by the same stream with potential-matching rows
  (Sec. 4.5, Eq. bc_both, md_bc): both evolve with the factor exp(-(i k.U + mu (k^2 + pi^2/4)) t);
  the discrete midpoint rule (Algorithm 1; a linear problem, so f' = 0 makes it plain RK2) gives
  the amplification (1 + lam dt + (lam dt)^2 / 2) per step;
* a steady Euler cellular flow (single-mode stream function, omega a multiple of psi): its
  convective term u.grad u is a gradient, so the curls in RHS_Omega2 and RHS_phi2 (Eq. om, phi)
  vanish while every C_ij is O(1);
* the plane-mean Reynolds-stress divergence of a single Fourier mode with a closed-form <u v>
  (Eq. mean_m1m3);
* the advection term of R_z at variable density, at the collocation points, where the product is
  exact (Sec. 2.1);
* a flat and an oblique diffusing interface of the binary-mixing fluid (Sec. 5): 1/rho is linear in
  z, and continuity plus the z equation give the exact curl-free momentum m^c = -kappa a rho grad z
  (a = (rho_h - rho_l)/(rho_l rho_h)) and dz/dt = kappa (lap z / rho + a |grad z|^2). The start-up
  fixed point (Sec. 3.1, Eq. y_k; reading R6) converged to rounding must reproduce both: this pins
  f'(z), rho_t = f' dz/dt, the m^c solve and the mean m^c solve (Eq. mc_mean), and the tail
  -(grad z / rho) . m^c of L (Sec. 4.3);
* the same flat interface translating with a uniform stream: momentum rho U gives
  d<m1>/dt = U rho_t (pins C_ij = -m_i m_j / rho and u = m / rho at variable density).

Each of these fails under a one-token sign or index change of the oracle line it pins.
"""
import numpy as np
import pytest

from oracle import banded
from oracle.lmvd import Config, Substage, _ax0
from oracle.transforms import padded_shape


def zero_state(S):
    cfg = S.cfg
    nxh = cfg.nx // 2 + 1
    z = np.zeros((cfg.ny, cfg.nz, nxh), complex)
    return dict(z=z, om=z.copy(), m2=np.zeros((cfg.ny + 1, cfg.nz, nxh), complex),
                mm1=np.zeros(cfg.ny), mm3=np.zeros(cfg.ny))


def coef_B(S, f):
    """Order-p coefficients of a y-profile by collocation at its Greville points."""
    return banded.solve(S.op.A_interp, f(S.op.basis.g).astype(complex))


def coef_Bs(S, f):
    """Order-(p+1) coefficients (the m2 space) by collocation at its Greville points."""
    return np.linalg.solve(S.op.basis.Ss[0], f(S.op.basis.gs).astype(complex))


def mixing_rho(cfg):
    """Binary-mixing fluid of Sec. 5: 1/rho = 1/rho_l - a z, a = (rho_h - rho_l) / (rho_l rho_h)."""
    a = (cfg.rho_h - cfg.rho_l) / (cfg.rho_l * cfg.rho_h)
    return a, (lambda z: 1.0 / (1.0 / cfg.rho_l - a * z))


def rhs_at(S, zdot):
    """RHS of Eq. DNS_system for the current state with m^c from a given dz/dt."""
    S.physical_pass_1()
    mc = S.mc_from_rhot(S.rho_t(zdot))
    F = S.physical_pass_2(mc)
    return S.rhs(F), mc


# ---- advection by a uniform stream (constant density) -----------------------------------------

def test_scalar_mode_in_uniform_stream():
    """z = eps exp(i(k1 x + k3 z)), uniform in y, m = (U, 0, W): dz/dt = -(i k.U + kappa k^2) z exactly."""
    cfg = Config(nx=8, ny=9, nz=8, rho_h=1.0, rho_l=1.0, re=100.0, dt=1e-3, n_startup=2, bc="potential")
    S = Substage(cfg)
    st = zero_state(S)
    U, W, eps = 0.7, -0.4, 1e-3
    jz, kx = 1, 2                      # kz = 1, kx = 2
    st["z"][:, jz, kx] = eps          # constant coefficients: a y-uniform profile
    st["mm1"][:] = U
    st["mm3"][:] = W
    S.set_state(**st)
    S.advance_substage()
    zdot = S.trace["zdot"]
    k1, k3 = 2.0, 1.0
    want = -(1j * (k1 * U + k3 * W) + (k1 ** 2 + k3 ** 2) / (cfg.re * cfg.sc)) * eps
    err = zdot.copy()
    err[:, jz, kx] -= want
    assert np.abs(err).max() < 1e-13 * abs(want)


@pytest.mark.parametrize("field", ["om", "m2"])
def test_vorticity_and_phi2_modes_in_uniform_stream(field):
    """Squire / Orr-Sommerfeld modes of a uniform stream under potential matching.

    Omega2 = eps sin(pi (y+1)/2) e^{i k.x} (Dirichlet rows), or m2^d with phi2 = eps sin(pi (y+1)/2) e^{i k.x}:
    m2 = c [s(y) + pi/(2k) e^{-k} cosh(k y)], c = -1/(pi^2/4 + k^2), which meets the Robin rows
    k m2 -+ m2' = 0 at y = -+1 and phi2(+-1) = 0. Both are advected and damped with
    lam = -(i k.U + mu (k^2 + pi^2/4)); the midpoint rule multiplies them by 1 + lam dt + (lam dt)^2/2.
    """
    cfg = Config(nx=8, ny=33, nz=8, rho_h=1.0, rho_l=1.0, re=10.0, dt=1e-3, n_startup=2, bc="potential")
    S = Substage(cfg)
    st = zero_state(S)
    U, W = 3.0, 1.0
    jz, kx = 2, 1                      # kz = 2, kx = 1: k.U = 5
    k1, k3 = 1.0, 2.0
    k = np.hypot(k1, k3)
    st["mm1"][:] = U
    st["mm3"][:] = W
    eps = 1e-8

    def s(y):
        return np.sin(np.pi * (y + 1) / 2)
    if field == "om":
        st["om"][:, jz, kx] = eps * coef_B(S, s)
    else:
        c = -1.0 / (np.pi ** 2 / 4 + k ** 2)
        st["m2"][:, jz, kx] = eps * coef_Bs(S, lambda y: c * (s(y) + np.pi / (2 * k) * np.exp(-k) * np.cosh(k * y)))
    S.set_state(**st)
    a0 = getattr(S, field)[:, jz, kx].copy()
    nsteps = 40
    S.step(nsteps)
    lam = -(1j * (k1 * U + k3 * W) + (k ** 2 + np.pi ** 2 / 4) / cfg.re)
    amp = (1 + lam * cfg.dt + (lam * cfg.dt) ** 2 / 2) ** nsteps
    a1 = getattr(S, field)[:, jz, kx]
    assert np.abs(a1 - a0 * amp).max() < 1e-6 * np.abs(a0).max()
    # the stream itself is a steady solution: Neumann rows, no shear
    assert np.abs(S.mm1 - U).max() < 1e-12 and np.abs(S.mm3 - W).max() < 1e-12


# ---- convective part of the RHS --------------------------------------------------------------

def test_steady_euler_cellular_flow_has_no_curl():
    """psi = cos(k s) sin(pi (y+1)/2), s along (k1, 0, k3)/k: a steady Euler flow (omega = lam psi).

    Its convective term d_j(u_i u_j) is a pressure gradient, so at mu = 0 the curls
    RHS_Omega2 = d3 H1 - d1 H3 and RHS_phi2 = lap H2 - d2 div H vanish, and so do the plane-mean
    stresses (<u v> = <w v> = 0). Every C_ij of this flow is O(1): u1 = (k1/k) u_s, u3 = (k3/k) u_s, k1 != k3.
    The remaining error is the spline representation of the sine profile (ny = 65).
    """
    cfg = Config(nx=16, ny=65, nz=16, rho_h=1.0, rho_l=1.0, re=1e300, dt=1e-3, n_startup=1)
    S = Substage(cfg)
    st = zero_state(S)
    k1, k3 = 1.0, 2.0
    k = np.hypot(k1, k3)
    # v = -d psi/ds = k sin(k s) S(y): Fourier coefficient -i k S(y) / 2 at (k1, k3)
    st["m2"][:, 2, 1] = -0.5j * k * coef_Bs(S, lambda y: np.sin(np.pi * (y + 1) / 2))
    S.set_state(**st)
    (r_om, r_phi, r_m1, r_m3), mc = rhs_at(S, np.zeros_like(S.z))
    assert np.abs(mc[1]).max() == 0.0                                  # f' = 0
    F = S.physical_pass_2(mc)
    for name in ("C11", "C12", "C13", "C22", "C23", "C33"):
        assert np.abs(F[name]).max() > 0.1, name                       # every stress takes part
    assert np.abs(r_om).max() < 1e-12
    assert np.abs(r_phi).max() < 1e-4        # terms are O(k^3 C) ~ 25; spline error ~3e-6 at ny = 65
    assert np.abs(r_m1).max() < 1e-14 and np.abs(r_m3).max() < 1e-14


def test_mean_reynolds_stress_divergence():
    """m2^d = A b(y) e^{i k x}, b = (1 - y^2) + i y (1 - y^2), Omega2 = 0: m1^d = i A b' / k and
    <u1 v> = 2 A^2 Re(i b' conj b) / k = -2 A^2 (1 - y^2)^2 / k, so RHS_<m1> = -d<u1 v>/dy
    = -8 A^2 y (1 - y^2) / k at mu = 0 (Eq. mean_m1m3). The same mode along z gives RHS_<m3>.
    Every profile is a polynomial inside the spline spaces, so the values at the collocation
    points are exact to rounding."""
    cfg = Config(nx=8, ny=17, nz=8, rho_h=1.0, rho_l=1.0, re=1e300, dt=1e-3, n_startup=1)
    S = Substage(cfg)
    st = zero_state(S)
    A1, A3 = 0.3, 0.2
    bc = coef_Bs(S, lambda y: (1 - y ** 2) + 1j * y * (1 - y ** 2))
    st["m2"][:, 0, 1] = A1 * bc                     # (kx, kz) = (1, 0)
    st["m2"][:, 2, 0] = A3 * bc                     # (0, 2) and its Hermitian partner (0, -2)
    st["m2"][:, cfg.nz - 2, 0] = np.conj(A3 * bc)
    S.set_state(**st)
    (r_om, r_phi, r_m1, r_m3), _ = rhs_at(S, np.zeros_like(S.z))
    g = S.op.basis.g
    w1 = -8 * A1 ** 2 * g * (1 - g ** 2) / 1.0
    w3 = -8 * A3 ** 2 * g * (1 - g ** 2) / 2.0
    assert np.abs(r_m1 - w1).max() < 1e-14 * np.abs(w1).max() * 10
    assert np.abs(r_m3 - w3).max() < 1e-14 * np.abs(w3).max() * 10


# ---- R_z at variable density ------------------------------------------------------------------

def test_rz_advection_and_diffusion_at_collocation_points():
    """z = z0(y) (cubic), m2^d = d (1 - y^2)^2 e^{i x}, density ratio 3: at the Greville points
    R_z = (-m2 z0' + kappa z0'') / rho exactly (Sec. 2.1, Eq. zeqn_imp), mode by mode."""
    cfg = Config(nx=8, ny=17, nz=8, rho_h=1.0, rho_l=1.0 / 3.0, re=100.0, dt=1e-3, n_startup=2)
    S = Substage(cfg)
    st = zero_state(S)

    def z0(y):
        return 0.5 + 0.3 * (y - y ** 3 / 3)

    def z1(y):
        return 0.3 * (1 - y ** 2)

    def z2(y):
        return -0.6 * y
    st["z"][:, 0, 0] = coef_B(S, z0)
    d = 1e-3
    st["m2"][:, 0, 1] = d * coef_Bs(S, lambda y: (1 - y ** 2) ** 2)
    S.set_state(**st)
    S.physical_pass_1()
    _, rho = mixing_rho(cfg)
    g = S.op.basis.g
    kappa = 1.0 / (cfg.re * cfg.sc)
    vals = _ax0(S.op.Bg[0], S.Rz)
    w1 = -d * (1 - g ** 2) ** 2 * z1(g) / rho(z0(g))
    w0 = kappa * z2(g) / rho(z0(g))
    assert np.abs(vals[:, 0, 1] - w1).max() < 1e-13 * np.abs(w1).max()
    assert np.abs(vals[:, 0, 0] - w0).max() < 1e-12 * np.abs(w0).max()
    other = vals.copy()
    other[:, 0, :2] = 0
    assert np.abs(other).max() < 1e-16


# ---- L, f' and m^c: diffusing interfaces of the binary-mixing fluid ---------------------------

def flat_interface(ny, **kw):
    cfg = Config(nx=4, ny=ny, nz=4, rho_h=1.0, rho_l=1.0 / 3.0, re=100.0, dt=1e-3, n_startup=80, **kw)
    S = Substage(cfg)
    st = zero_state(S)
    # z0' = 0.3 (1 - y^2) vanishes at both walls: the exact m2^c then meets <m2^c>(+1) = 0
    st["z"][:, 0, 0] = coef_B(S, lambda y: 0.5 + 0.3 * (y - y ** 3 / 3))
    return S, st


def test_flat_diffusing_interface_exact_momentum():
    """z = z0(y): the start-up fixed point gives <m2^c> = -kappa a rho z0' and
    dz/dt = kappa (z0'' / rho + a z0'^2) (continuity + the z equation with 1/rho linear in z)."""
    S, st = flat_interface(65)
    S.set_state(**st)
    cfg = S.cfg
    assert S.startup_residuals[-1] < 1e-14
    a, rho = mixing_rho(cfg)
    kappa = 1.0 / (cfg.re * cfg.sc)
    gs, g = S.op.basis.gs, S.op.basis.g

    def z0(y):
        return 0.5 + 0.3 * (y - y ** 3 / 3)

    def z1(y):
        return 0.3 * (1 - y ** 2)
    mc = S.mc_from_rhot(S.rho_t(S.zdot0))
    m2 = np.real(S.op.basis.Ss[0] @ mc[1][:, 0, 0])
    want_m2 = -kappa * a * rho(z0(gs)) * z1(gs)
    assert np.abs(m2 - want_m2).max() < 1e-9 * np.abs(want_m2).max()
    zd = np.real(S.op.basis.Bg[0] @ S.zdot0[:, 0, 0])
    want_zd = kappa * (-0.6 * g / rho(z0(g)) + a * z1(g) ** 2)
    assert np.abs(zd - want_zd).max() < 1e-9 * np.abs(want_zd).max()
    assert np.abs(S.zdot0[:, :, 1:]).max() == 0 and np.abs(S.zdot0[:, 1:, :]).max() == 0


def test_oblique_diffusing_interface_exact_momentum():
    """z = 1/2 + 1/5 cos(x + 2z), uniform in y: m^c = -kappa a rho grad z (curl free: a function of
    x + 2z times a fixed vector) and dz/dt = kappa (lap z / rho + a |grad z|^2), on the padded grid.
    The x and z components have different weights, so swapping them fails. 1/rho has geometrically
    decaying harmonics that the 32 x 64 grid resolves to rounding."""
    cfg = Config(nx=32, ny=8, nz=64, rho_h=1.0, rho_l=1.0 / 3.0, re=100.0, dt=1e-3, n_startup=80)
    S = Substage(cfg)
    st = zero_state(S)
    st["z"][:, 0, 0] = 0.5
    st["z"][:, 2, 1] = 0.1            # 0.2 cos(theta) = 0.1 e^{i theta} + c.c., theta = x + 2z
    S.set_state(**st)
    assert S.startup_residuals[-1] < 1e-14
    a, rho_of = mixing_rho(cfg)
    kappa = 1.0 / (cfg.re * cfg.sc)
    px, pz = padded_shape(cfg.nx, cfg.nz)
    X, Z = np.meshgrid(2 * np.pi * np.arange(px) / px, 2 * np.pi * np.arange(pz) / pz)
    th = X + 2 * Z
    zf, zx, zz, lap = 0.5 + 0.2 * np.cos(th), -0.2 * np.sin(th), -0.4 * np.sin(th), -1.0 * np.cos(th)
    rho = rho_of(zf)
    want_zd = kappa * (lap / rho + a * (zx ** 2 + zz ** 2))
    op = S.op
    zd = op.phys(_ax0(op.Bg[0], S.zdot0))
    assert np.abs(zd - want_zd[None]).max() < 1e-13 * np.abs(want_zd).max()
    m1, m2, m3 = S.mc_from_rhot(S.rho_t(S.zdot0))
    p1 = op.phys(_ax0(op.Bg[0], m1))
    p3 = op.phys(_ax0(op.Bg[0], m3))
    w1, w3 = -kappa * a * rho * zx, -kappa * a * rho * zz
    assert np.abs(p1 - w1[None]).max() < 1e-13 * np.abs(w1).max()
    assert np.abs(p3 - w3[None]).max() < 1e-13 * np.abs(w3).max()
    assert np.abs(m2).max() < 1e-16


def test_translating_flat_interface_momentum_rate():
    """<m1> = rho(y) U, <m3> = rho(y) W on the flat interface: u = (U, 0, W) has no shear, and the
    momentum changes only because rho does: d<m1>/dt = U rho_t, d<m3>/dt = W rho_t with
    rho_t = kappa a rho (z0'' + a rho z0'^2) (Eq. mean_m1m3 with C_ij = -m_i m_j / rho, u = m / rho)."""
    S, st = flat_interface(65, bc="potential")
    cfg = S.cfg
    a, rho = mixing_rho(cfg)
    kappa = 1.0 / (cfg.re * cfg.sc)
    U, W = 0.6, -0.25

    def z0(y):
        return 0.5 + 0.3 * (y - y ** 3 / 3)
    st["mm1"] = np.real(coef_B(S, lambda y: U * rho(z0(y))))
    st["mm3"] = np.real(coef_B(S, lambda y: W * rho(z0(y))))
    S.set_state(**st)
    assert S.startup_residuals[-1] < 1e-14
    (r_om, r_phi, r_m1, r_m3), _ = rhs_at(S, S.zdot0)
    g = S.op.basis.g
    r = rho(z0(g))
    rho_t = kappa * a * r * (-0.6 * g + a * r * (0.3 * (1 - g ** 2)) ** 2)
    assert np.abs(r_m1 - U * rho_t).max() < 1e-7 * np.abs(U * rho_t).max()
    assert np.abs(r_m3 - W * rho_t).max() < 1e-7 * np.abs(W * rho_t).max()
