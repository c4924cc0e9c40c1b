"""Algorithm 1 (segregated RK2 with incomplete fixed-point iteration) on the scalar test system.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper Sec. 3.3 (system ODE) and Sec. 3.3.1 (temporal convergence tests):
  dz/dt  = M1(z) dz/dt + M2(z),     M1 = c1 (1 + sin z),  M2 = c2 exp(z)
  dm^d/dt = M3(m^d, m^c) = c3 m^d (m^c)^3
  d rho/dt = G(m^c) = c4 m^c,       rho = f(z) = z
with c1 = 0.6i, c2 = -1, c3 = 2 - 0.8i, c4 = -3 + 0.5i, z0 = m^d_0 = 0.5.
Guesses from Eq. dzdt_guesses (beta^n = 0, beta' = -4 by default), k_f iterations
of Eq. y_k, m^c = G^{-1}(f'(z) dz/dt), midpoint RK2 in low-storage form.
Reference: dz/dt = M2 / (1 - M1) integrated directly (Sec. 3.3.1).
Start-up (not given in the paper): dz/dt^0 from the exact inverse of (1 - M1),
history back-filled by Taylor steps (Appendix A expansions truncated at O(dt)).
"""
import numpy as np

C1, C2, C3, C4 = 0.6j, -1.0 + 0j, 2.0 - 0.8j, -3.0 + 0.5j


def M1(z):
    return C1 * (1 + np.sin(z))


def M2(z):
    return C2 * np.exp(z)


def M3(md, mc):
    return C3 * md * mc ** 3


def stage_coefficients(s, beta_n, beta_p):
    """Guess coefficients of Eq. dzdt_guesses (dt dz/dt^0 = a0 z^s + a1 z^{s-1} + a2 z^{s-2} + a3 z^{s-3})
    and the low-storage RK2 weights (alpha, beta) of substage s (even: stage n, odd: stage ')."""
    if s % 2 == 0:
        return (2.0, -(2.0 + 0.5 * beta_n), beta_n, -0.5 * beta_n), (0.5, 0.0)
    return (4.0 + beta_p, -(5.0 + 2.0 * beta_p), beta_p, 1.0), (1.0, -0.5)


def zdot_of_substage(s, z, hist, dt, kf, beta_n, beta_p, m1=None, m2=None):
    """dz/dt^{s,k_f}: the guess of Eq. dzdt_guesses from z and its history hist = [z^{s-1}, z^{s-2},
    z^{s-3}], then kf applications of the fixed point of Eq. y_k, dz/dt <- M1(z) dz/dt + M2(z)."""
    m1 = M1 if m1 is None else m1
    m2 = M2 if m2 is None else m2
    a, _ = stage_coefficients(s, beta_n, beta_p)
    g = (a[0] * z + a[1] * hist[0] + a[2] * hist[1] + a[3] * hist[2]) / dt
    for _ in range(kf):
        g = m1(z) * g + m2(z)
    return g


def run(dt, t_end, kf=4, beta_n=0.0, beta_p=-4.0, z0=0.5 + 0j, md0=0.5 + 0j):
    """Return (z, m^d) at t_end after round(t_end/dt) RK2 steps of Algorithm 1."""
    nsteps = int(round(t_end / dt))
    z, md = complex(z0), complex(md0)
    zdot = M2(z) / (1 - M1(z))
    hist = [z - 0.5 * dt * zdot, z - dt * zdot, z - 1.5 * dt * zdot]   # z^{s-1}, z^{s-2}, z^{s-3}
    zdot_prev, r_prev = zdot, 0j
    for s in range(2 * nsteps):
        _, (al, be) = stage_coefficients(s, beta_n, beta_p)
        g = zdot_of_substage(s, z, hist, dt, kf, beta_n, beta_p)
        mc = g / C4                      # G^{-1}(f'(z) dz/dt) with f' = 1
        r = M3(md, mc)
        z_new = z + dt * (al * g + be * zdot_prev)
        md_new = md + dt * (al * r + be * r_prev)
        hist = [z, hist[0], hist[1]]
        zdot_prev, r_prev = g, r
        z, md = z_new, md_new
    return z, md


def reference(t_end, z0=0.5 + 0j, md0=0.5 + 0j):
    """(z, m^d) at t_end from dz/dt = M2/(1 - M1), m^c = (dz/dt)/c4, integrated with DOP853."""
    from scipy.integrate import solve_ivp

    def f(t, y):
        z = y[0] + 1j * y[1]
        md = y[2] + 1j * y[3]
        zd = M2(z) / (1 - M1(z))
        mdd = M3(md, zd / C4)
        return [zd.real, zd.imag, mdd.real, mdd.imag]

    sol = solve_ivp(f, (0.0, t_end), [z0.real, z0.imag, md0.real, md0.imag], method="DOP853",
                    rtol=1e-13, atol=1e-15)
    y = sol.y[:, -1]
    return y[0] + 1j * y[1], y[2] + 1j * y[3]
