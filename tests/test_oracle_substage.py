"""Pins for oracle/lmvd.py against identities and closed forms the paper and the mathematics fix.

* m^d is exactly divergence free and reproduces Omega2 (Sec. 4.1, Eq. md_recon);
* m^c satisfies mass conservation exactly in B-coefficient space, the curl-free equation at its
  collocation points and its boundary rows (Sec. 4.2, Eq. COM_fourier, CF_fourier, mc_mean);
* the k-th fixed-point iterate has error L^k (y^0 - y) (Sec. 3.1, Eq. y_k_delta);
* the BDF-like guess coefficients satisfy the Taylor conditions of Appendix A;
* constant density: m^c = 0, dz/dt = R_z = kappa lap z; Stokes decay of a mean shear mode, of an
  Omega2 mode and of an m2^d mode at the closed-form rates (KMM limit, Sec. 1.3);
* gravity drives heavy-over-light unstable and light-over-heavy stable (Sec. 5);
* the full substage sequence converges at second order in dt (Sec. 3.3).
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import banded
from oracle.lmvd import Config, Substage, _ax0


def zero_state(S):
    cfg = S.cfg
    nxh = cfg.nx // 2 + 1
    z = np.zeros((cfg.ny, cfg.nz, nxh), complex)
    return dict(z=z, om=z.copy(), m2=np.zeros((cfg.ny + 1, cfg.nz, nxh), complex),
                mm1=np.zeros(cfg.ny), mm3=np.zeros(cfg.ny))


def interp_profile(S, f):
    """B coefficients of a y-profile by collocation at the Greville points."""
    return banded.solve(S.op.A_interp, f(S.op.basis.g).astype(complex))


def rt_like(cfg, eps_eta=0.02, width=0.1, seed=0, vel=1e-3):
    """Small RT-shaped state for tests (tanh interface with a few modes, small velocity)."""
    S = Substage(cfg)
    rng = np.random.default_rng(seed)
    st = zero_state(S)
    nx, nz = cfg.nx, cfg.nz
    x = 2 * np.pi * np.arange(nx) / nx
    zc = 2 * np.pi * np.arange(nz) / nz
    eta = eps_eta * (np.cos(x[None, :] + 0.3) + 0.5 * np.cos(x[None, :] + zc[:, None] + 1.1))
    g = S.op.basis.g
    rh, rl = cfg.rho_h, cfg.rho_l
    rho = 0.5 * (rh + rl) + 0.5 * (rh - rl) * np.tanh((g[:, None, None] - eta[None]) / width)
    zf = rh / (rh - rl) * (1 - rl / rho) if rh != rl else np.zeros_like(rho)
    zh = np.fft.rfft2(zf, axes=(1, 2), norm="forward")
    zh[:, nz // 2] = 0
    zh[:, :, nx // 2] = 0
    st["z"] = banded.solve(S.op.A_interp, zh)
    ys = S.op.basis.gs
    prof = (1 - ys ** 2) ** 2
    for (jz, kx) in ((0, 1), (1, 1), (nz - 1, 1)):
        st["m2"][:, jz, kx] = vel * complex(rng.normal(), rng.normal()) * prof
        st["om"][:, jz, kx] = vel * complex(rng.normal(), rng.normal()) * (1 - g ** 2)
    st["m2"][[1, cfg.ny - 1]] = 0
    return S, st


@pytest.fixture(scope="module")
def rt8():
    cfg = Config(nx=8, ny=13, nz=8, rho_l=1 / 3, re=200.0, dt=2e-3, n_startup=10)
    S, st = rt_like(cfg)
    S.set_state(**st)
    return S


def test_md_divergence_free_and_vorticity(rt8):
    S = rt8
    op = S.op
    m1, m3 = S.md_components(S.m2, S.om, S.mm1, S.mm3)
    div = 1j * op.k1 * m1 + 1j * op.k3 * m3 + _ax0(op.D, S.m2)
    assert np.abs(div).max() < 1e-15 * max(1.0, np.abs(S.m2).max() * 100)
    om = (1j * op.k3 * m1 - 1j * op.k1 * m3) * op.kmask
    assert np.abs(om - S.om).max() < 1e-14 * np.abs(S.om).max()


def test_mc_mass_curlfree_and_bcs(rt8):
    S = rt8
    op = S.op
    ny = S.cfg.ny
    rng = np.random.default_rng(5)
    rt = S.rho_t(rng.normal(size=S.z.shape) * op.keep)
    m1, m2, m3 = S.mc_from_rhot(rt)
    # mass conservation holds without discretisation error in B-coefficient space
    res = S.mass_residual(rt, (m1, m2, m3))
    assert np.abs(res).max() < 1e-13 * np.abs(rt).max()
    # curl-free equation at the interior B* Greville points: d m_par/dy - i k m2 = 0
    k = np.sqrt(op.k2)
    mpar = np.where(op.kmask, (op.k1 * m1 + op.k3 * m3) / np.where(op.kmask, k, 1), 0)
    cf = _ax0(op.Bs[1], mpar) - 1j * k * _ax0(op.Ss[0], m2)
    assert np.abs(cf[1:ny] * op.kmask).max() < 1e-12 * np.abs(mpar).max() * ny
    # second curl-free constraint k3 m1 - k1 m3 = 0
    assert np.abs(op.k3 * m1 - op.k1 * m3).max() < 1e-15 * max(1, np.abs(m1).max())
    # walls: m2^c(+-1) = 0 for k != 0; plane mean vanishes at the top wall, <m1^c> = <m3^c> = 0
    tol = 1e-14 * np.abs(m2).max()     # pivoting solves reach the BC rows only up to rounding
    assert np.abs(m2[0] * op.kmask).max() < tol and np.abs(m2[ny] * op.kmask).max() < tol
    assert abs(m2[ny, 0, 0]) < tol and np.abs(m1[:, 0, 0]).max() == 0 and np.abs(m3[:, 0, 0]).max() == 0


def test_fixed_point_error_is_L_power_times_initial_error():
    """Eq. y_k_delta: y^k = y + L^k (y^0 - y), y the exact fixed point (tiny grid, L built densely)."""
    cfg = Config(nx=4, ny=9, nz=4, rho_l=1 / 3, re=200.0, dt=2e-3, n_startup=2)
    S, st = rt_like(cfg, eps_eta=0.05, width=0.2)
    S.set_state(**st)
    S.physical_pass_1()
    keep = S.op.keep
    idx = np.nonzero(np.broadcast_to(keep, S.z.shape).ravel())[0]

    def vec(c):
        f = c.ravel()[idx]
        return np.concatenate([f.real, f.imag])

    def unvec(v):
        c = np.zeros(S.z.size, complex)
        c[idx] = v[:len(idx)] + 1j * v[len(idx):]
        return c.reshape(S.z.shape)

    n = 2 * len(idx)
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = vec(S.apply_L(unvec(e)))
    b = vec(S.Rz)
    # restrict to the Hermitian-consistent subspace spanned by L's range plus b
    y_star, *_ = np.linalg.lstsq(np.eye(n) - L, b, rcond=None)
    assert np.abs((np.eye(n) - L) @ y_star - b).max() < 1e-12 * np.abs(b).max()
    y = vec(S.bdf_guess())
    y0 = y.copy()
    for k in range(1, 5):
        y = vec(S.apply_L(unvec(y)) + S.Rz)
        pred = y_star + np.linalg.matrix_power(L, k) @ (y0 - y_star)
        assert np.abs(y - pred).max() < 1e-11 * np.abs(y_star).max()


def test_bdf_coefficients_taylor_conditions():
    """Appendix A: the guesses reproduce dt z'(t_n) (stage n) and dt z'(t_n) + dt^2/2 z''(t_n) (stage ')."""
    cfg = Config(nx=4, ny=9, nz=4, dt=1.0)
    S = Substage(cfg)
    one = np.ones((1,))
    cases = {
        0: ([0.0, -0.5, -1.0, -1.5], [0.0, 0.0, 0.5, 1.0], 1.0, 0.0),   # z^n, z^{n-1,'}, z^{n-1}, z^{n-2,'}
        1: ([0.5, 0.0, -0.5, -1.0], [0.0, 0.0, 0.0, 0.5], 1.0, 0.5),    # z', z^n, z^{n-1,'}, z^{n-1}
    }
    for s, (c1, c2, want1, want2) in cases.items():
        S.s = s
        for beta in (0.0, -4.0, 1.7):
            S.cfg.beta_n = S.cfg.beta_p = beta
            S.z, S.zh = one, [one * 0, one * 0, one * 0]
            S.z = one * 1.0
            S.zh = [one * 1.0, one * 1.0, one * 1.0]
            assert abs(S.bdf_guess()[0]) < 1e-14                           # constants -> 0
            S.z, S.zh = one * c1[0], [one * c1[1], one * c1[2], one * c1[3]]
            assert abs(S.bdf_guess()[0] - want1) < 1e-14                   # dt z' term
            S.z, S.zh = one * c2[0], [one * c2[1], one * c2[2], one * c2[3]]
            assert abs(S.bdf_guess()[0] - want2) < 1e-14                   # dt^2 z'' term


def const_density_cfg(**kw):
    base = dict(nx=4, ny=33, nz=4, rho_h=1.0, rho_l=1.0, re=10.0, dt=1e-3, n_startup=2)
    base.update(kw)
    return Config(**base)


def test_constant_density_zdot_is_diffusion():
    cfg = const_density_cfg(ny=17)
    S = Substage(cfg)
    st = zero_state(S)
    eps = 1e-3
    st["z"][:, 0, 1] = eps / 2                                    # z = eps cos(x), uniform in y
    st["z"][:, 0, 0] = interp_profile(S, lambda y: 0.25 * np.cos(np.pi * y))
    S.set_state(**st)
    S.advance_substage()
    zdot = S.trace["zdot"]
    kappa = 1.0 / cfg.re
    want = np.zeros_like(zdot)
    want[:, 0, 1] = -kappa * eps / 2
    want[:, 0, 0] = interp_profile(S, lambda y: -kappa * np.pi ** 2 * 0.25 * np.cos(np.pi * y))
    assert np.abs(S.trace["mc"][1]).max() == 0.0                  # f' = 0 -> m^c = 0
    assert np.abs(zdot[:, 0, 1] - want[:, 0, 1]).max() < 1e-15
    # the y-profile part carries the O(h^4) collocation error of d2/dy2 cos(pi y) at ny = 17
    assert np.abs(zdot[:, 0, 0] - want[:, 0, 0]).max() < 1e-3 * kappa * np.pi ** 2 * 0.25


def _decay_run(S, st, nsteps, getter):
    S.set_state(**st)
    a0 = getter(S)
    S.step(nsteps)
    return getter(S), a0


def test_mean_shear_decay_closed_form():
    cfg = const_density_cfg()
    S = Substage(cfg)
    st = zero_state(S)
    st["mm1"] = np.real(interp_profile(S, lambda y: np.cos(np.pi * y / 2)))
    nsteps = 50
    a1, a0 = _decay_run(S, st, nsteps, lambda S: S.mm1.copy())
    rate = (np.pi / 2) ** 2 / cfg.re
    assert np.abs(a1 - a0 * np.exp(-rate * nsteps * cfg.dt)).max() < 1e-7 * np.abs(a0).max()


def test_omega2_stokes_mode_decay():
    cfg = const_density_cfg()
    S = Substage(cfg)
    st = zero_state(S)
    eps = 1e-8
    st["om"][:, 0, 1] = eps * interp_profile(S, lambda y: np.sin(np.pi * (y + 1) / 2))
    nsteps = 50
    a1, a0 = _decay_run(S, st, nsteps, lambda S: S.om[:, 0, 1].copy())
    rate = (1.0 + (np.pi / 2) ** 2) / cfg.re
    assert np.abs(a1 - a0 * np.exp(-rate * nsteps * cfg.dt)).max() < 1e-7 * np.abs(a0).max()


def test_m2d_stokes_mode_decay():
    """Even no-slip Stokes mode v = cos(qy) - cos(q)/cosh(k) cosh(ky), q tan q = -k tanh k."""
    cfg = const_density_cfg(ny=33)
    S = Substage(cfg)
    op = S.op
    k = 1.0
    q = brentq(lambda q: q * np.tan(q) + k * np.tanh(k), np.pi / 2 + 1e-9, np.pi - 1e-9)

    def v(y):
        return np.cos(q * y) - np.cos(q) / np.cosh(k) * np.cosh(k * y)
    ny = cfg.ny
    A = op.Amd2.copy()
    A[2:ny - 1] = op.basis.Ss[0][2:ny - 1]
    rhs = np.zeros(ny + 1)
    rhs[2:ny - 1] = v(op.basis.gs[2:ny - 1])
    st = zero_state(S)
    st["m2"][:, 0, 1] = 1e-8 * np.linalg.solve(A, rhs)
    nsteps = 50
    a1, a0 = _decay_run(S, st, nsteps, lambda S: S.m2[:, 0, 1].copy())
    rate = (k * k + q * q) / cfg.re
    assert np.abs(a1 - a0 * np.exp(-rate * nsteps * cfg.dt)).max() < 1e-6 * np.abs(a0).max()


@pytest.mark.parametrize("heavy_on_top", [True, False])
def test_gravity_sign(heavy_on_top):
    """A raised interface (eta > 0 at x = 0) rises further when heavy fluid is on top, sinks back otherwise."""
    rh, rl = (1.0, 1.0 / 3.0) if heavy_on_top else (1.0 / 3.0, 1.0)
    cfg = Config(nx=4, ny=33, nz=4, rho_h=rh, rho_l=rl, re=1000.0, dt=1e-3, n_startup=10)
    S = Substage(cfg)
    st = zero_state(S)
    x = 2 * np.pi * np.arange(4) / 4
    g = S.op.basis.g
    eta = 0.02 * np.cos(x)[None, :] * np.ones((4, 1))
    rho = 0.5 * (rh + rl) + 0.5 * (rh - rl) * np.tanh((g[:, None, None] - eta[None]) / 0.1)
    zf = rh / (rh - rl) * (1 - rl / rho)
    zh = np.fft.rfft2(zf, axes=(1, 2), norm="forward")
    zh[:, 2] = 0
    zh[:, :, 2] = 0
    st["z"] = banded.solve(S.op.A_interp, zh)
    S.set_state(**st)
    S.step(3)
    m2_mid = S.m2[cfg.ny // 2 + 1, 0, 1]
    assert abs(m2_mid.imag) < 1e-6 * abs(m2_mid.real)
    assert (m2_mid.real > 0) == heavy_on_top


def test_hermitian_and_mass_over_substages(rt8):
    S = rt8
    for _ in range(3):
        S.advance_substage()
        res = S.mass_residual(S.trace["rho_t"], S.trace["mc"])
        assert np.abs(res).max() < 1e-13 * max(1e-30, np.abs(S.trace["rho_t"]).max())
        for f in (S.z, S.om):
            col = f[:, :, 0]
            nz = S.cfg.nz
            for jz in range(1, nz // 2):
                assert np.abs(col[:, jz] - np.conj(col[:, nz - jz])).max() < 1e-15 * max(1, np.abs(col).max())


@pytest.mark.slow
def test_second_order_in_time_full_substage():
    """Self-convergence of the whole scheme on a small RT-shaped state: error ratio -> 4 per halving."""
    out = []
    T = 0.024
    for dt in (4e-3, 2e-3, 1e-3, 5e-4):
        cfg = Config(nx=8, ny=17, nz=8, rho_l=1 / 3, re=200.0, dt=dt, n_startup=60)
        S, st = rt_like(cfg, vel=1e-2)
        S.set_state(**st)
        S.step(int(round(T / dt)))
        out.append((S.z.copy(), S.m2.copy(), S.om.copy()))
    for f in range(3):
        e1 = np.linalg.norm(out[0][f] - out[1][f])
        e2 = np.linalg.norm(out[1][f] - out[2][f])
        e3 = np.linalg.norm(out[2][f] - out[3][f])
        assert 3.2 < e1 / e2 < 4.8 and 3.2 < e2 / e3 < 4.8, (f, e1 / e2, e2 / e3)
