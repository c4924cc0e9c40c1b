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
