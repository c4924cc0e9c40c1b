"""Fourier transforms in the two periodic directions with the 3/2 rule (paper Eq. disc_f, Sec. 4.4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Spectral arrays have shape (ny, nz, nx//2 + 1), complex: axis 1 is kz in FFT order
(slot j -> kz = j for j < nz/2, j - nz for j > nz/2), axis 2 is kx = 0 .. nx/2.
Only |kx| < nx/2 and |kz| < nz/2 are retained (Eq. disc_f sums to N/2 - 1); the
Nyquist slots kx = nx/2 and kz = nz/2 are always zero.
Physical arrays have shape (ny, pz, px) with px = 3 nx / 2, pz = 3 nz / 2: the
padded grid on which products are formed (3/2-rule dealiasing).
Normalisation: f(x, z) = sum_k fhat_k exp(i k.x) (unscaled synthesis), so the
analysis carries 1 / (px pz).
scipy.fft (pocketfft) is the transform primitive, run with one worker per host core.
"""
import os

import numpy as np
import scipy.fft as sfft

WORKERS = os.cpu_count() or 1


def padded_shape(nx, nz):
    if nx % 2 or nz % 2:
        raise ValueError("nx and nz must be even")
    return 3 * nx // 2, 3 * nz // 2


def to_phys(fhat, nx, nz):
    """Spectral (ny, nz, nx/2+1) -> physical (ny, pz, px) on the 3/2-padded grid."""
    px, pz = padded_shape(nx, nz)
    ny = fhat.shape[0]
    w = np.zeros((ny, pz, px // 2 + 1), dtype=np.complex128)
    h = nz // 2
    w[:, :h, :nx // 2] = fhat[:, :h, :nx // 2]                   # kz = 0 .. nz/2 - 1
    w[:, pz - h + 1:, :nx // 2] = fhat[:, h + 1:, :nx // 2]      # kz = -nz/2 + 1 .. -1
    return sfft.irfft2(w, s=(pz, px), axes=(1, 2), norm="forward", workers=WORKERS)


def to_spec(f, nx, nz):
    """Physical (ny, pz, px) -> spectral (ny, nz, nx/2+1), truncated, Nyquist zero."""
    px, pz = padded_shape(nx, nz)
    assert f.shape[1:] == (pz, px)
    w = sfft.rfft2(f, axes=(1, 2), norm="forward", workers=WORKERS)
    out = np.zeros((f.shape[0], nz, nx // 2 + 1), dtype=np.complex128)
    h = nz // 2
    out[:, :h, :nx // 2] = w[:, :h, :nx // 2]
    out[:, h + 1:, :nx // 2] = w[:, pz - h + 1:, :nx // 2]
    return out


def wavenumbers(nx, nz, lx, lz):
    """k1, k3 arrays of shape (nz, nx/2+1) for the spectral layout (Nyquist slots carry 0)."""
    kx = 2 * np.pi / lx * np.arange(nx // 2 + 1, dtype=np.float64)
    kx[nx // 2] = 0.0
    jz = np.arange(nz)
    kz = 2 * np.pi / lz * np.where(jz < nz // 2, jz, jz - nz).astype(np.float64)
    kz[nz // 2] = 0.0
    k1 = np.broadcast_to(kx[None, :], (nz, nx // 2 + 1)).copy()
    k3 = np.broadcast_to(kz[:, None], (nz, nx // 2 + 1)).copy()
    return k1, k3


def retained_mask(nx, nz):
    """True where a mode is retained (all but the Nyquist row and column)."""
    m = np.ones((nz, nx // 2 + 1), dtype=bool)
    m[nz // 2, :] = False
    m[:, nx // 2] = False
    return m
