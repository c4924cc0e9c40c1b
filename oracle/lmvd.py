"""One substage of the variable-density pseudospectral method, written step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows the paper:
  Sec. 2  (Eq. mom_decomp, COMass, COMom; the operators L and R_z, Eq. zeqn_imp),
  Sec. 3  (incomplete fixed-point iteration Eq. y_k; BDF-like guesses Eq. dzdt_guesses;
           segregated RK2, Algorithm 1),
  Sec. 4  (Fourier representation Eq. disc_f; m^d from Eq. phi_poisson / md_recon;
           m^c from Eq. COM_fourier, CF_fourier, mc_recon, mc_mean; applying L (Sec. 4.3);
           the DNS system Eq. DNS_system and its time advance, Algorithm 2),
  Appendix A (coefficients of the guesses), Appendix C (B-spline spaces, exact D*),
  Sec. 5  (Rayleigh-Taylor physics: gravity, the binary-mixing equation of state).

Readings of points the paper leaves open:
  R1 Nyquist modes kx = nx/2, kz = nz/2 are zero; products are formed on the 3/2 grid.
  R2 B-spline order p (default 6) for all fields but m2; order p+1 for m2; clamped
     uniform knots; collocation at Greville abscissae of the order-p space for values,
     at Greville abscissae of the order-(p+1) space for the m2 equations.
  R3 mass conservation holds in B-coefficient space through the exact bidiagonal D*;
     the curl-free equation is collocated at the interior order-(p+1) Greville points.
  R4 bc = "walls": no-slip walls at y = +-1 replace potential matching: Omega2 = 0;
     m2^d = d m2^d/dy = 0; m2^c = 0; <m1> = <m3> = 0; dz/dy = 0; <m2^c>(+1) = 0.
     bc = "potential": the paper's own conditions (Sec. 4.5, Eq. bc_both, md_bc): the Robin
     rows k m2 -+ dm2/dy = 0 at y = -1 / +1 (Eq. bc_both times k) for m2^c and m2^d;
     phi2 = 0 at both ends (Eq. md_bc) as the two remaining m2^d rows; Omega2 = 0;
     d<m1>/dy = d<m3>/dy = 0; dz/dy = 0; <m2^c>(+1) = 0. The m1, m3 lines of Eq. bc_both
     are not imposed separately: they follow from Omega2 = 0 and the Robin row for m^d,
     and from the curl-free construction for m^c wherever rho_t vanishes at the boundary.
  R5 the state holds the B* coefficients of m2^d instead of phi2 = (D^2 - k^2) m2^d;
     phi2 is that operator collocated at the order-(p+1) Greville points 2 .. ny-2.
  R6 start-up: n_startup fixed-point iterations from dz/dt = 0, then the history
     z^{s-1}, z^{s-2}, z^{s-3} is back-filled by Taylor steps with that dz/dt.
  R7 k_f applications of L per stage, starting from the BDF-like guess.
  R8 rho_h = 1, rho_l = 1/ratio, mu = 1/Re, rho D_z = 1/(Re Sc), gravity 1/Fr^2 along -y.
  R9 RK2 is the midpoint rule in low-storage form:
     X^{s+1} = X^s + dt (alpha_s R^s + beta_s R^{s-1}), (alpha, beta) = (1/2, 0), (1, -1/2).
  R10 the viscous stress term (1/3) grad(div u) cancels in both curls and is dropped.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import banded
from .bspline import Basis
from .transforms import padded_shape, retained_mask, to_phys, to_spec, wavenumbers


@dataclass
class Config:
    nx: int
    ny: int
    nz: int
    p: int = 6
    lx: float = 2 * np.pi
    lz: float = 2 * np.pi
    y0: float = -1.0
    y1: float = 1.0
    re: float = 1000.0
    sc: float = 1.0
    fr: float = 1.0
    rho_h: float = 1.0
    rho_l: float = 1.0 / 3.0
    dt: float = 1e-3
    kf: int = 4
    beta_n: float = 0.0
    beta_p: float = -4.0
    n_startup: int = 20
    bc: str = "walls"          # "walls" | "potential" (reading R4)


def _ax0(op, F):
    """Apply a y-operator (rows x ny) along axis 0 of F."""
    out = op @ F.reshape(F.shape[0], -1)
    return np.asarray(out).reshape((op.shape[0],) + F.shape[1:])


class Operators:
    """All y-matrices and wavenumbers of one configuration (Appendix C)."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        ny = cfg.ny
        b = Basis(ny, cfg.p, cfg.y0, cfg.y1)
        self.basis = b
        csr = sp.csr_matrix
        self.Bg = [csr(m) for m in b.Bg]   # B^(d) at g   (ny x ny)
        self.Bs = [csr(m) for m in b.Bs]   # B^(d) at g*  ((ny+1) x ny)
        self.Sg0 = csr(b.Sg[0])            # B* at g      (ny x (ny+1))
        self.Ss = [csr(m) for m in b.Ss]   # B*^(d) at g* ((ny+1) x (ny+1))
        self.D = csr(b.D)                  # D*           (ny x (ny+1))
        # interpolation / Dirichlet matrix: values at g (rows 0, ny-1 are the wall values)
        self.A_interp = b.Bg[0].copy()
        # Neumann matrix for z: wall rows replaced by dz/dy at y = -1, +1
        An = b.Bg[0].copy()
        An[0, :] = b.Bg[1][0, :]
        An[ny - 1, :] = b.Bg[1][ny - 1, :]
        self.A_neumann = An
        potential = cfg.bc == "potential"
        if cfg.bc not in ("walls", "potential"):
            raise ValueError("bc must be 'walls' or 'potential'")
        # The per-mode matrices are A(k) = A2 - k^2 A0 + k A1. Potential matching (Eq. bc_both
        # times k): row 0: k m2(-1) - dm2/dy(-1) = 0, row ny: k m2(+1) + dm2/dy(+1) = 0.
        # (g*_0 = -1 and g*_ny = +1: clamped knots put the end Greville points on the boundary.)
        def robin(A2, A0, A1):
            for r, sgn in ((0, -1.0), (ny, 1.0)):
                A2[r, :] = sgn * b.Ss[1][r, :]
                A0[r, :] = 0.0
                A1[r, :] = b.Ss[0][r, :]
        # m^c system (Eq. COM_fourier + CF_fourier, eliminated for m2^c):
        #   rows 1..ny-1: (B*'' - k^2 B*)(g*_i) m2 = -B'(g*_i) rho_t;
        #   rows 0, ny: walls m2(-1) = m2(+1) = 0, or the Robin rows
        A2 = b.Ss[2].copy()
        A0 = b.Ss[0].copy()
        A1 = np.zeros_like(A2)
        for r in (0, ny):
            A2[r, :] = 0.0
            A2[r, r] = 1.0
            A0[r, :] = 0.0
        if potential:
            robin(A2, A0, A1)
        self.Amc2, self.Amc0, self.Amc1 = A2, A0, A1
        # m2^d update (Eq. phi_poisson): rows 2..ny-2: (B*'' - k^2 B*)(g*_i) m2 = phi2-target;
        #   walls: m2(+-1) = dm2/dy(+-1) = 0 in rows 0, ny and 1, ny-1;
        #   potential: Robin rows 0, ny; phi2(-1) = 0 in row 1 and phi2(+1) = 0 in row ny-1 (Eq. md_bc)
        A2 = b.Ss[2].copy()
        A0 = b.Ss[0].copy()
        A1 = np.zeros_like(A2)
        for r in (0, 1, ny - 1, ny):
            A0[r, :] = 0.0
            A2[r, :] = 0.0
        if potential:
            robin(A2, A0, A1)
            A2[1, :] = b.Ss[2][0, :]
            A0[1, :] = b.Ss[0][0, :]
            A2[ny - 1, :] = b.Ss[2][ny, :]
            A0[ny - 1, :] = b.Ss[0][ny, :]
        else:
            A2[0, 0] = 1.0
            A2[ny, ny] = 1.0
            A2[1, :] = b.Ss[1][0, :]
            A2[ny - 1, :] = b.Ss[1][ny, :]
        self.Amd2, self.Amd0, self.Amd1 = A2, A0, A1
        # plane means <m1>, <m3>: Dirichlet rows (walls) or Neumann rows (potential matching)
        self.A_means = self.A_neumann if potential else self.A_interp
        # plane-mean m2^c (Eq. mc_mean): D* c = -<rho_t>, c(+1) = 0
        Am = np.zeros((ny + 1, ny + 1))
        Am[:ny, :] = b.D
        Am[ny, ny] = 1.0
        self.A_mcmean = Am

        self.k1, self.k3 = wavenumbers(cfg.nx, cfg.nz, cfg.lx, cfg.lz)
        self.k2 = self.k1 ** 2 + self.k3 ** 2
        self.keep = retained_mask(cfg.nx, cfg.nz)
        self.kmask = self.keep & (self.k2 > 0)   # retained modes with k != 0
        self.mu = 1.0 / cfg.re
        self.kappa = 1.0 / (cfg.re * cfg.sc)
        self.grav = 1.0 / cfg.fr ** 2

    # ---- helpers -----------------------------------------------------------------
    def spec(self, rows):
        return np.zeros((rows, self.cfg.nz, self.cfg.nx // 2 + 1), dtype=np.complex128)

    def interp(self, V):
        """B-spline coefficients from values at g (collocation solve)."""
        return banded.solve(self.A_interp, V) * self.keep

    def phys(self, F):
        return to_phys(F, self.cfg.nx, self.cfg.nz)

    def spectral(self, f):
        return to_spec(f, self.cfg.nx, self.cfg.nz)

    def solve_k2(self, A2, A0, rhs, A1=None):
        """Per-mode solve of (A2 - k^2 A0 + k A1) x = rhs over the modes with k != 0."""
        out = np.zeros_like(rhs)
        idx = np.nonzero(self.kmask.ravel())[0]
        r = rhs.reshape(rhs.shape[0], -1)
        o = out.reshape(rhs.shape[0], -1)
        o[:, idx] = banded.solve_k2(A2, A0, self.k2.ravel()[idx], r[:, idx], A1)
        return out


class Substage:
    """State and the six steps of Algorithm 2 for one configuration."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.op = Operators(cfg)
        self.s = 0
        self.trace = {}

    # ---- Sec. 4.1: divergence-free momentum ---------------------------------------
    def md_components(self, m2, om, mm1, mm3):
        """Eq. md_recon: m1^d, m3^d (B coefficients) from m2^d (B*) and Omega2 (B); k = 0 from the means."""
        op = self.op
        dm2 = _ax0(op.D, m2)
        k1, k3, k2 = op.k1, op.k3, op.k2
        safe = np.where(op.kmask, k2, 1.0)
        m1 = np.where(op.kmask, (1j * k1 * dm2 - 1j * k3 * om) / safe, 0)
        m3 = np.where(op.kmask, (1j * k3 * dm2 + 1j * k1 * om) / safe, 0)
        m1[:, 0, 0] = mm1
        m3[:, 0, 0] = mm3
        return m1, m3

    # ---- Sec. 4.2: curl-free momentum from rho_t ----------------------------------
    def mc_from_rhot(self, rt):
        """Eq. COM_fourier, CF_fourier, mc_recon, mc_mean: (m1^c, m2^c (B*), m3^c) from rho_t (B coefs)."""
        op = self.op
        ny = self.cfg.ny
        rhs = op.spec(ny + 1)
        rhs[1:ny] = -_ax0(op.Bs[1], rt)[1:ny]
        m2 = op.solve_k2(op.Amc2, op.Amc0, rhs, op.Amc1)
        # plane mean: D* <m2^c> = -<rho_t>, <m2^c>(+1) = 0
        b = np.zeros(ny + 1, dtype=np.complex128)
        b[:ny] = -rt[:, 0, 0]
        m2[:, 0, 0] = np.linalg.solve(op.A_mcmean, b)
        k = np.sqrt(op.k2)
        safe = np.where(op.kmask, k, 1.0)
        mpar = np.where(op.kmask, 1j * (rt + _ax0(op.D, m2)) / safe, 0)
        m1 = np.where(op.kmask, op.k1 / safe * mpar, 0)
        m3 = np.where(op.kmask, op.k3 / safe * mpar, 0)
        return m1, m2, m3

    # ---- physical-space pieces (Sec. 2.1, 4.3, 5) ---------------------------------
    def eos(self, z):
        """rho = rho_l rho_h / (rho_h - (rho_h - rho_l) z) and f'(z) = d rho / d z (Sec. 5)."""
        rh, rl = self.cfg.rho_h, self.cfg.rho_l
        den = rh - (rh - rl) * z
        return rl * rh / den, rl * rh * (rh - rl) / den ** 2

    def rho_t(self, zdot):
        """rho_t = f'(z) dz/dt formed in physical space, returned as B coefficients (Sec. 4.3)."""
        op = self.op
        return op.interp(op.spectral(self.fprime * op.phys(_ax0(op.Bg[0], zdot))))

    def apply_L_tail(self, mc):
        """-(1/rho) grad z . m^c formed in physical space, returned as B coefficients (Sec. 4.3)."""
        op = self.op
        m1, m2, m3 = mc
        p1 = op.phys(_ax0(op.Bg[0], m1))
        p2 = op.phys(_ax0(op.Sg0, m2))
        p3 = op.phys(_ax0(op.Bg[0], m3))
        return op.interp(op.spectral(-(self.w[0] * p1 + self.w[1] * p2 + self.w[2] * p3)))

    def apply_L(self, zdot):
        """L(z){zdot} (Sec. 4.3): rho_t = f' zdot -> m^c = C(rho_t) -> -(1/rho) grad z . m^c."""
        return self.apply_L_tail(self.mc_from_rhot(self.rho_t(zdot)))

    # ---- step 1 + step 2 of Algorithm 2 -------------------------------------------
    def physical_pass_1(self):
        """m^d, z and its derivatives in physical space; rho, f', grad z / rho, R_z (Sec. 2.1)."""
        op = self.op
        cfg = self.cfg
        m1d, m3d = self.md_components(self.m2, self.om, self.mm1, self.mm3)
        zg = _ax0(op.Bg[0], self.z)
        zyg = _ax0(op.Bg[1], self.z)
        zyyg = _ax0(op.Bg[2], self.z)
        zp = op.phys(zg)
        zx = op.phys(1j * op.k1 * zg)
        zz = op.phys(1j * op.k3 * zg)
        zy = op.phys(zyg)
        lapz = op.phys(-op.k2 * zg + zyyg)
        self.md_phys = (op.phys(_ax0(op.Bg[0], m1d)), op.phys(_ax0(op.Sg0, self.m2)), op.phys(_ax0(op.Bg[0], m3d)))
        rho, fp = self.eos(zp)
        self.rho, self.fprime = rho, fp
        self.w = (zx / rho, zy / rho, zz / rho)
        u1, u2, u3 = self.md_phys
        rz = (-(u1 * zx + u2 * zy + u3 * zz) + op.kappa * lapz) / rho
        self.Rz = op.interp(op.spectral(rz))
        self.trace.update(m1d=m1d, m3d=m3d, Rz=self.Rz)
        _ = cfg

    def bdf_guess(self):
        """Eq. dzdt_guesses: dt dz/dt^{s,0} from z^s, z^{s-1}, z^{s-2}, z^{s-3} (Appendix A)."""
        cfg = self.cfg
        if self.s % 2 == 0:   # stage n
            bn = cfg.beta_n
            a = (2.0, -(2.0 + 0.5 * bn), bn, -0.5 * bn)
        else:                 # stage ' (t_{n+1/2})
            bp = cfg.beta_p
            a = (4.0 + bp, -(5.0 + 2.0 * bp), bp, 1.0)
        return (a[0] * self.z + a[1] * self.zh[0] + a[2] * self.zh[1] + a[3] * self.zh[2]) / cfg.dt

    # ---- step 5: RHS of Eq. DNS_system ---------------------------------------------
    def physical_pass_2(self, mc):
        """m = m^d + m^c, u = m / rho, C_ij = -rho u_i u_j (Eq. om, phi), as B coefficients."""
        op = self.op
        m1c, m2c, m3c = mc
        mcp = (op.phys(_ax0(op.Bg[0], m1c)), op.phys(_ax0(op.Sg0, m2c)), op.phys(_ax0(op.Bg[0], m3c)))
        m = [self.md_phys[i] + mcp[i] for i in range(3)]
        rho = self.rho
        out = {}
        for (i, j) in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)):
            out["C%d%d" % (i + 1, j + 1)] = op.interp(op.spectral(-m[i] * m[j] / rho))
        for i in range(3):
            out["u%d" % (i + 1)] = op.interp(op.spectral(m[i] / rho))
        out["rho"] = op.interp(op.spectral(rho))
        return out

    def rhs(self, F):
        """RHS_Omega2 (at g), RHS_phi2 (at g*), RHS_<m1>, RHS_<m3> (at g), Eq. DNS_system.

        H_i = d_j C_ij + mu lap u_i - g rho delta_i2 (constant mu; the (1/3) grad div u part of
        d_j tau_ij is a gradient and cancels in both curls);
        RHS_Omega2 = d3 H1 - d1 H3;  RHS_phi2 = lap H2 - d2 (d_j H_j) = -k^2 H2 - d2 (i k1 H1 + i k3 H3).
        """
        op = self.op
        k1, k3, k2 = op.k1, op.k3, op.k2
        mu, g = op.mu, op.grav

        def at_g(name, d):
            return _ax0(op.Bg[d], F[name])

        def at_s(name, d):
            return _ax0(op.Bs[d], F[name])

        # H1, H3 at g; Omega2 RHS
        lap_u1 = -k2 * at_g("u1", 0) + at_g("u1", 2)
        lap_u3 = -k2 * at_g("u3", 0) + at_g("u3", 2)
        H1 = 1j * k1 * at_g("C11", 0) + at_g("C12", 1) + 1j * k3 * at_g("C13", 0) + mu * lap_u1
        H3 = 1j * k1 * at_g("C13", 0) + at_g("C23", 1) + 1j * k3 * at_g("C33", 0) + mu * lap_u3
        r_om = (1j * k3 * H1 - 1j * k1 * H3) * op.kmask
        # at g*: H2 and d/dy of (i k1 H1 + i k3 H3)
        H2 = (1j * k1 * at_s("C12", 0) + at_s("C22", 1) + 1j * k3 * at_s("C23", 0)
              + mu * (-k2 * at_s("u2", 0) + at_s("u2", 2)) - g * at_s("rho", 0))
        dH1 = (1j * k1 * at_s("C11", 1) + at_s("C12", 2) + 1j * k3 * at_s("C13", 1)
               + mu * (-k2 * at_s("u1", 1) + at_s("u1", 3)))
        dH3 = (1j * k1 * at_s("C13", 1) + at_s("C23", 2) + 1j * k3 * at_s("C33", 1)
               + mu * (-k2 * at_s("u3", 1) + at_s("u3", 3)))
        r_phi = (-k2 * H2 - (1j * k1 * dH1 + 1j * k3 * dH3)) * op.kmask
        # plane means (Eq. mean_m1m3): d/dy (<C12> + mu d<u1>/dy), d/dy (<C23> + mu d<u3>/dy)
        r_m1 = np.real(at_g("C12", 1)[:, 0, 0] + mu * at_g("u1", 2)[:, 0, 0])
        r_m3 = np.real(at_g("C23", 1)[:, 0, 0] + mu * at_g("u3", 2)[:, 0, 0])
        return r_om, r_phi, r_m1, r_m3

    # ---- step 6: RK2 update ----------------------------------------------------------
    def rk_coeffs(self):
        return (0.5, 0.0) if self.s % 2 == 0 else (1.0, -0.5)

    def update(self, zdot, R):
        """Midpoint RK2 in low-storage form at the collocation points, then the BC-row solves."""
        op = self.op
        cfg = self.cfg
        ny, dt = cfg.ny, cfg.dt
        al, be = self.rk_coeffs()
        r_om, r_phi, r_m1, r_m3 = R
        p_om, p_phi, p_m1, p_m3 = self.Rprev
        # Omega2: interior values advanced, Dirichlet rows
        v = _ax0(op.Bg[0], self.om) + dt * (al * r_om + be * p_om)
        v[0] = 0
        v[ny - 1] = 0
        om = banded.solve(op.A_interp, v) * op.kmask
        # plane means: interior values advanced; Dirichlet (walls) or Neumann (potential) rows
        mm = []
        for cur, r, pr in ((self.mm1, r_m1, p_m1), (self.mm3, r_m3, p_m3)):
            v = op.Bg[0] @ cur + dt * (al * r + be * pr)
            v[0] = 0
            v[ny - 1] = 0
            mm.append(banded.solve(op.A_means, v))
        # z: interior values advanced with dz/dt^{k_f}, Neumann rows
        v = _ax0(op.Bg[0], self.z + dt * (al * zdot + be * self.zdot_prev))
        v[0] = 0
        v[ny - 1] = 0
        z = banded.solve(op.A_neumann, v) * op.keep
        # m2^d: phi2 at g*_2..g*_{ny-2} advanced, four boundary rows (no-slip or potential matching)
        phi = _ax0(op.Ss[2], self.m2) - op.k2 * _ax0(op.Ss[0], self.m2)
        v = phi + dt * (al * r_phi + be * p_phi)
        v[:2] = 0
        v[ny - 1:] = 0
        m2 = op.solve_k2(op.Amd2, op.Amd0, v, op.Amd1)
        return z, om, m2, mm[0], mm[1]

    # ---- public API ------------------------------------------------------------------
    def set_state(self, z, om, m2, mm1, mm3, history=None):
        op = self.op
        self.z = np.array(z, dtype=np.complex128) * op.keep
        self.om = np.array(om, dtype=np.complex128) * op.kmask
        self.m2 = np.array(m2, dtype=np.complex128) * op.kmask
        self.mm1 = np.array(mm1, dtype=np.float64)
        self.mm3 = np.array(mm3, dtype=np.float64)
        self.s = 0
        if history is not None:
            self.s = int(history["s"])
            self.zh = [np.array(history[k], dtype=np.complex128) for k in ("z1", "z2", "z3")]
            self.zdot_prev = np.array(history["zdot"], dtype=np.complex128)
            self.Rprev = (np.array(history["r_om"]), np.array(history["r_phi"]),
                          np.array(history["r_m1"]), np.array(history["r_m3"]))
            return
        self.startup()

    def startup(self):
        """Reading R6: n_startup fixed-point iterations from dz/dt = 0, Taylor back-fill of the history."""
        cfg = self.cfg
        self.physical_pass_1()
        zdot = np.zeros_like(self.z)
        res = []
        for _ in range(cfg.n_startup):
            new = self.apply_L(zdot) + self.Rz
            res.append(np.linalg.norm(new - zdot) / max(np.linalg.norm(new), 1e-300))
            zdot = new
        self.startup_residuals = res
        self.zdot0 = zdot
        dt = cfg.dt
        self.zh = [self.z - 0.5 * dt * zdot, self.z - dt * zdot, self.z - 1.5 * dt * zdot]
        self.zdot_prev = zdot.copy()
        op = self.op
        self.Rprev = (op.spec(cfg.ny), op.spec(cfg.ny + 1), np.zeros(cfg.ny), np.zeros(cfg.ny))

    def history(self):
        return dict(s=self.s, z1=self.zh[0], z2=self.zh[1], z3=self.zh[2], zdot=self.zdot_prev,
                    r_om=self.Rprev[0], r_phi=self.Rprev[1], r_m1=self.Rprev[2], r_m3=self.Rprev[3])

    def state(self):
        return dict(z=self.z, om=self.om, m2=self.m2, mm1=self.mm1, mm3=self.mm3)

    def advance_substage(self):
        """Algorithm 2, steps 1-6, for substage s -> s+1."""
        cfg = self.cfg
        # steps 1-2: m^d, R_z, rho, f', grad z / rho; BDF-like guess
        self.physical_pass_1()
        zdot = self.bdf_guess()
        self.trace["zdot_guess"] = zdot
        # step 3: k_f fixed-point iterations of Eq. y_k, then m^c from dz/dt^{k_f}
        res = []
        for _ in range(cfg.kf):
            new = self.apply_L(zdot) + self.Rz
            res.append(np.linalg.norm(new - zdot) / max(np.linalg.norm(new), 1e-300))
            zdot = new
        rt = self.rho_t(zdot)
        mc = self.mc_from_rhot(rt)
        self.fp_residuals = res
        self.trace.update(zdot=zdot, rho_t=rt, mc=mc)
        # steps 4-5: properties from z^s (rho held from pass 1), RHS
        F = self.physical_pass_2(mc)
        R = self.rhs(F)
        self.trace.update(F=F, R=R)
        # step 6: RK2 update and history rotation
        z, om, m2, mm1, mm3 = self.update(zdot, R)
        self.zh = [self.z, self.zh[0], self.zh[1]]
        self.zdot_prev = zdot
        self.Rprev = R
        self.z, self.om, self.m2, self.mm1, self.mm3 = z, om, m2, mm1, mm3
        self.s += 1

    def step(self, n):
        for _ in range(2 * n):
            self.advance_substage()

    # ---- diagnostics ------------------------------------------------------------------
    def mass_residual(self, rt, mc):
        """rho_t + i k1 m1^c + i k3 m3^c + D* m2^c in B-coefficient space (zero up to rounding)."""
        op = self.op
        m1, m2, m3 = mc
        return rt + 1j * op.k1 * m1 + 1j * op.k3 * m3 + _ax0(op.D, m2)
