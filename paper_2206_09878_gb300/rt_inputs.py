"""Seeded synthetic Rayleigh-Taylor-shaped initial states.

This module holds none of the method's arithmetic: no B-spline evaluation, no
collocation solve, no padded transform, no product of the method. It writes
B-spline coefficient arrays directly, using the fact that a spline whose
coefficients are samples of a smooth profile at nearby abscissae is a smooth
approximation of that profile (a variation-diminishing quasi-interpolant). The
abscissae are the generator's own uniform points, not the method's collocation
points. The only transform is numpy's unpadded rfft2 of a sampled field, which
projects the sampled interface onto Fourier modes.

Recipe (all arrays use the spectral layout [y][kz][kx], kx = 0..nx/2, kz in FFT
order, Nyquist slots zero):
  rho  = (rho_h + rho_l)/2 + (rho_h - rho_l)/2 tanh((y - eta(x, z)) / width)
         heavy fluid on top, rho_h = 1, rho_l = 1 / ratio;
  eta  = sum_k a cos(kx x + kz z + theta_k) over integer (kx, kz) with
         0 < kx^2 + kz^2 <= kmax^2, one of each +- pair, theta_k ~ U[0, 2 pi)
         from numpy.random.default_rng(seed), a rescaled so rms(eta) = eta_rms;
  z    = rho_h / (rho_h - rho_l) (1 - rho_l / rho)   (binary-mixing variable);
  m2^d = c_k (1 - y^2)^2, Omega2 = d_k (1 - y^2) on the same wavenumber band,
         c_k, d_k complex normal from default_rng(seed + 1000), Hermitian on
         kx = 0; the two coefficients next to each wall of m2^d are zero so the
         no-slip conditions hold; both are rescaled so the sampled rms of m2^d
         and of Omega2 / |k| equal u_rms;
  <m1> = <m3> = 0.

The paper's own single-mode set-up (Sec. 5, its domains V^{3D,1}, V^{3D,2} with W = 1, g = 1) is
PAPER_RT / rt_paper_state: potential-matching boundaries (bc_mode 1) on [0, 1] x [y0, y1] x [0, 1];
  z   = (1 + tanh((y - h) / (2 eps))) / 2,  eps = 0.05,
  h   = 0.05 (cos 2 pi x + cos 2 pi z) + delta  (3D; delta = 0 on [-2, 2], 0.5 on [-3.5, 3.5]),
  rho_h = 1, rho_l = (1 - At) / (1 + At), Re = 1024, Sc = 1, Fr = 1, dt = 2.5e-4 / sqrt(At);
  the paper's initial momentum m = -(1/(Re Sc)) grad rho is a gradient, so its divergence-free
  part is zero: Omega2 = m2^d = <m1> = <m3> = 0, and the curl-free part is what the method's
  start-up derives from rho_t. The "+ delta" the paper also prints after the z profile is read as
  part of h only (z must stay in [0, 1]).
"""
import numpy as np

# (nx, ny, nz, ratio, width, kmax, eta_rms, u_rms, re, dt, steps, seed)
WORKLOADS = {
    "rt32": dict(nx=32, ny=33, nz=32, ratio=3.0, width=0.05, kmax=4, eta_rms=1e-2, u_rms=1e-4,
                 re=1000.0, dt=1e-3, steps=5, seed=1001),
    "rt128": dict(nx=128, ny=129, nz=128, ratio=3.0, width=0.05, kmax=8, eta_rms=1e-2, u_rms=1e-4,
                  re=1000.0, dt=5e-4, steps=20, seed=1004),
    "rt256": dict(nx=256, ny=257, nz=256, ratio=25.7, width=0.02, kmax=16, eta_rms=5e-3, u_rms=1e-4,
                  re=3000.0, dt=2e-4, steps=20, seed=1002),
    "rt512": dict(nx=512, ny=513, nz=512, ratio=10.0, width=0.05, kmax=32, eta_rms=2e-3, u_rms=1e-4,
                  re=5000.0, dt=1e-4, steps=10, seed=1003),
    "rt768": dict(nx=768, ny=769, nz=768, ratio=25.7, width=0.02, kmax=48, eta_rms=1e-3, u_rms=1e-4,
                  re=8000.0, dt=2e-4 * 256 / 768, steps=5, seed=1005),
    # rt512 with 33 B-spline rows: the same transform lengths (768) for a small ncu capture
    "rt512y33": dict(nx=512, ny=33, nz=512, ratio=10.0, width=0.05, kmax=32, eta_rms=2e-3, u_rms=1e-4,
                     re=5000.0, dt=1e-4, steps=1, seed=1003),
}


def _band_modes(nx, nz, kmax):
    """(kx, kz) integer pairs with 0 < kx^2 + kz^2 <= kmax^2, one of each +- pair."""
    out = []
    for kx in range(0, min(kmax, nx // 2 - 1) + 1):
        for kz in range(-min(kmax, nz // 2 - 1), min(kmax, nz // 2 - 1) + 1):
            if kx == 0 and kz <= 0:
                continue
            if 0 < kx * kx + kz * kz <= kmax * kmax:
                out.append((kx, kz))
    return out


def rt_state(nx, ny, nz, ratio, width, kmax, eta_rms, u_rms, seed, **_):
    """Return dict(z, om, m2, mm1, mm3) of numpy arrays (complex128 / float64)."""
    rh, rl = 1.0, 1.0 / ratio
    nxh = nx // 2 + 1
    x = 2 * np.pi * np.arange(nx) / nx
    zc = 2 * np.pi * np.arange(nz) / nz
    rng = np.random.default_rng(seed)
    modes = _band_modes(nx, nz, kmax)
    theta = rng.uniform(0.0, 2 * np.pi, size=len(modes))
    eta = np.zeros((nz, nx))
    for (kx, kz), th in zip(modes, theta):
        eta += np.cos(kx * x[None, :] + kz * zc[:, None] + th)
    eta *= eta_rms / np.sqrt(np.mean(eta ** 2))

    y = -1.0 + 2.0 * np.arange(ny) / (ny - 1)           # the generator's own anchors
    rho = 0.5 * (rh + rl) + 0.5 * (rh - rl) * np.tanh((y[:, None, None] - eta[None]) / width)
    zfield = rh / (rh - rl) * (1.0 - rl / rho)
    zhat = np.fft.rfft2(zfield, axes=(1, 2), norm="forward")
    zhat[:, nz // 2, :] = 0
    zhat[:, :, nx // 2] = 0

    rng2 = np.random.default_rng(seed + 1000)
    ys = -1.0 + 2.0 * np.arange(ny + 1) / ny
    m2 = np.zeros((ny + 1, nz, nxh), dtype=np.complex128)
    om = np.zeros((ny, nz, nxh), dtype=np.complex128)
    prof2 = (1 - ys ** 2) ** 2
    prof2[[0, 1, ny - 1, ny]] = 0.0
    prof1 = 1 - y ** 2
    prof1[[0, ny - 1]] = 0.0
    kmag = []
    for (kx, kz) in modes:
        c = complex(rng2.normal(), rng2.normal())
        d = complex(rng2.normal(), rng2.normal())
        jz = kz % nz
        m2[:, jz, kx] = c * prof2
        om[:, jz, kx] = d * prof1
        if kx == 0:   # Hermitian partner of a kx = 0 mode
            m2[:, (-kz) % nz, 0] = np.conj(c) * prof2
            om[:, (-kz) % nz, 0] = np.conj(d) * prof1
        kmag.append(np.hypot(kx, kz))

    def rms(a, w):
        return np.sqrt(np.sum(w * np.abs(a) ** 2) / a.shape[0])

    wts = np.full((nz, nxh), 2.0)
    wts[:, 0] = 1.0
    kk = np.hypot(np.arange(nxh)[None, :], np.where(np.arange(nz) < nz // 2, np.arange(nz), np.arange(nz) - nz)[:, None])
    kk[0, 0] = 1.0
    m2 *= u_rms / max(rms(m2, wts), 1e-300)
    om *= u_rms / max(rms(om / kk, wts), 1e-300)
    return dict(z=zhat, om=om, m2=m2, mm1=np.zeros(ny), mm3=np.zeros(ny))


# The paper's case table (Table RT_casedetails, with the domains defined beside it), W = g = 1:
# domain name -> (y0, y1, mesh); (dimension, At) -> Reynolds number, domain, dt sqrt(At) / sqrt(W/g).
# The last 3D row prints the domain V^{2D,2}; as a 3D case it is read as V^{3D,2}.
PAPER_DOMAINS = {"2D,1": (-2.0, 2.0, (128, 512)), "2D,2": (-3.5, 3.5, (128, 1024)),
                 "3D,1": (-2.0, 2.0, (128, 512, 128)), "3D,2": (-3.5, 3.5, (128, 1024, 128))}
PAPER_CASES = {
    (2, 0.33): dict(re=3000.0, domain="2D,1", dt_scaled=2.5e-4),
    (2, 0.5): dict(re=3000.0, domain="2D,1", dt_scaled=2.5e-4),
    (2, 0.67): dict(re=3000.0, domain="2D,1", dt_scaled=2.5e-4),
    (2, 0.8): dict(re=3000.0, domain="2D,1", dt_scaled=2.5e-4),
    (2, 0.925): dict(re=3000.0, domain="2D,2", dt_scaled=1.25e-4),
    (3, 0.33): dict(re=1024.0, domain="3D,1", dt_scaled=2.5e-4),
    (3, 0.5): dict(re=1024.0, domain="3D,1", dt_scaled=2.5e-4),
    (3, 0.67): dict(re=1024.0, domain="3D,2", dt_scaled=1.25e-4),
    (3, 0.8): dict(re=1024.0, domain="3D,2", dt_scaled=6.25e-5),
    (3, 0.925): dict(re=1024.0, domain="3D,2", dt_scaled=3.125e-5),
}


def paper_dt(dim, at):
    """Time step of the paper's table for (dim, At): dt_scaled / sqrt(At). An At the table does not list
    takes the 2.5e-4 of its low-At rows."""
    row = PAPER_CASES.get((dim, round(float(at), 3)))
    return float((row["dt_scaled"] if row else 2.5e-4) / np.sqrt(at))


# the paper's 3D single-mode Rayleigh-Taylor cases (Sec. 5): (nx, ny, nz, At, y0, y1, delta, steps);
# rtp128 and rtp128_hi are the table's V^{3D,1} and V^{3D,2} meshes, rtp32 a small V^{3D,1} case
PAPER_RT = {
    "rtp32": dict(nx=32, ny=65, nz=32, at=0.5, y0=-2.0, y1=2.0, delta=0.0, steps=5),
    "rtp128": dict(nx=128, ny=512, nz=128, at=0.5, y0=-2.0, y1=2.0, delta=0.0, steps=10),
    "rtp128_hi": dict(nx=128, ny=1024, nz=128, at=0.8, y0=-3.5, y1=3.5, delta=0.5, steps=10),
}


def paper_rt_config(nx, ny, nz, at, y0, y1, **_):
    """Problem constants of the paper's 3D set-up (W = g = 1, Sc = 1; Re and dt from its case table)."""
    row = PAPER_CASES.get((3, round(float(at), 3)), dict(re=1024.0))
    return dict(nx=nx, ny=ny, nz=nz, lx=1.0, lz=1.0, y0=y0, y1=y1, re=row["re"], sc=1.0, fr=1.0, rho_h=1.0,
                rho_l=(1.0 - at) / (1.0 + at), dt=paper_dt(3, at), bc="potential")


def rt_paper_state(nx, ny, nz, y0, y1, delta, eps=0.05, **_):
    """dict(z, om, m2, mm1, mm3) of the paper's initial condition (module docstring)."""
    nxh = nx // 2 + 1
    x = np.arange(nx) / nx
    zc = np.arange(nz) / nz
    h = 0.05 * (np.cos(2 * np.pi * x)[None, :] + np.cos(2 * np.pi * zc)[:, None]) + delta
    y = y0 + (y1 - y0) * np.arange(ny) / (ny - 1)           # the generator's own anchors
    zfield = 0.5 * (1.0 + np.tanh((y[:, None, None] - h[None]) / (2 * eps)))
    zhat = np.fft.rfft2(zfield, axes=(1, 2), norm="forward")
    zhat[:, nz // 2, :] = 0
    zhat[:, :, nx // 2] = 0
    return dict(z=zhat, om=np.zeros((ny, nz, nxh), np.complex128), m2=np.zeros((ny + 1, nz, nxh), np.complex128),
                mm1=np.zeros(ny), mm3=np.zeros(ny))


def eta_modes(nx, nz, kmax, seed, **_):
    """The interface modes of rt_state: (kx, kz) pairs, their phases theta_k, and the amplitude a that
    rt_state gives every mode (the rms rescaling), as numpy arrays."""
    x = 2 * np.pi * np.arange(nx) / nx
    zc = 2 * np.pi * np.arange(nz) / nz
    rng = np.random.default_rng(seed)
    modes = _band_modes(nx, nz, kmax)
    theta = rng.uniform(0.0, 2 * np.pi, size=len(modes))
    eta = np.zeros((nz, nx))
    for (kx, kz), th in zip(modes, theta):
        eta += np.cos(kx * x[None, :] + kz * zc[:, None] + th)
    return np.array(modes), theta, np.sqrt(1.0 / np.mean(eta ** 2))


def z_from_eta_torch(amps, modes, theta, nx, ny, nz, ratio, width, **_):
    """z_hat of rt_state for eta = sum_k amps[k] cos(kx x + kz z + theta_k), written with torch operations
    so that it is differentiable in amps (a float64 tensor; the result lives on amps' device)."""
    import torch
    dev, f64 = amps.device, torch.float64
    rh, rl = 1.0, 1.0 / ratio
    x = 2 * np.pi * torch.arange(nx, dtype=f64, device=dev) / nx
    zc = 2 * np.pi * torch.arange(nz, dtype=f64, device=dev) / nz
    kx = torch.as_tensor(modes[:, 0], dtype=f64, device=dev)
    kz = torch.as_tensor(modes[:, 1], dtype=f64, device=dev)
    th = torch.as_tensor(theta, dtype=f64, device=dev)
    phase = kx[:, None, None] * x[None, None, :] + kz[:, None, None] * zc[None, :, None] + th[:, None, None]
    eta = (amps[:, None, None] * torch.cos(phase)).sum(0)
    y = -1.0 + 2.0 * torch.arange(ny, dtype=f64, device=dev) / (ny - 1)
    rho = 0.5 * (rh + rl) + 0.5 * (rh - rl) * torch.tanh((y[:, None, None] - eta[None]) / width)
    zfield = rh / (rh - rl) * (1.0 - rl / rho)
    zhat = torch.fft.rfft2(zfield, dim=(1, 2), norm="forward")
    keep = torch.ones(zhat.shape[1:], dtype=f64, device=dev)
    keep[nz // 2, :] = 0
    keep[:, nx // 2] = 0
    return zhat * keep
