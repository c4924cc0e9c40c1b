"""Pins for oracle/transforms.py (paper Eq. disc_f, 3/2-rule products): exact trig fields, brute force, Parseval."""
import numpy as np
import pytest

from oracle.transforms import padded_shape, retained_mask, to_phys, to_spec, wavenumbers


def grid(nx, nz):
    px, pz = padded_shape(nx, nz)
    x = 2 * np.pi * np.arange(px) / px
    z = 2 * np.pi * np.arange(pz) / pz
    return x[None, :], z[:, None]


def test_trig_field_coefficients_and_derivatives():
    nx, nz = 16, 12
    x, z = grid(nx, nz)
    f = np.cos(2 * x + 3 * z) + 0.5 * np.sin(x - 2 * z) + 0.25
    fh = to_spec(f[None], nx, nz)[0]
    exp = np.zeros_like(fh)
    exp[3, 2] = 0.5               # cos(2x+3z) = (e^{i(2x+3z)} + cc)/2
    exp[-2, 1] = -0.25j           # 0.5 sin(x-2z): coefficient of e^{i(x-2z)} is 0.5/(2i)
    exp[0, 0] = 0.25
    assert np.abs(fh - exp).max() < 1e-15
    k1, k3 = wavenumbers(nx, nz, 2 * np.pi, 2 * np.pi)
    dfx = to_phys((1j * k1 * fh)[None], nx, nz)[0]
    dfz = to_phys((1j * k3 * fh)[None], nx, nz)[0]
    assert np.abs(dfx - (-2 * np.sin(2 * x + 3 * z) + 0.5 * np.cos(x - 2 * z))).max() < 1e-13
    assert np.abs(dfz - (-3 * np.sin(2 * x + 3 * z) - np.cos(x - 2 * z))).max() < 1e-13


def _random_spec(rng, nx, nz, ny=1):
    """A random real band-limited field: build it in physical space on the unpadded grid."""
    f = rng.normal(size=(ny, nz, nx))
    fh = np.fft.rfft2(f, axes=(1, 2), norm="forward")
    fh[:, nz // 2, :] = 0
    fh[:, :, nx // 2] = 0
    return fh


def test_roundtrip_retained_modes():
    rng = np.random.default_rng(1)
    nx, nz = 16, 10
    fh = _random_spec(rng, nx, nz, ny=3)
    back = to_spec(to_phys(fh, nx, nz), nx, nz)
    assert np.abs(back - fh).max() < 1e-15
    assert not np.any(back[:, nz // 2, :]) and not np.any(back[:, :, nx // 2])


def test_dealiased_product_equals_truncated_convolution():
    """With the 3/2 rule, the product of two fields with |k| < N/2 has no aliasing (brute-force convolution)."""
    rng = np.random.default_rng(2)
    nx, nz = 8, 8
    ah, bh = _random_spec(rng, nx, nz)[0], _random_spec(rng, nx, nz)[0]
    prod = to_spec(to_phys(ah[None], nx, nz) * to_phys(bh[None], nx, nz), nx, nz)[0]

    def full(fh):   # dictionary (kx, kz) -> coefficient over all retained modes incl. kx < 0
        d = {}
        for jz in range(nz):
            kz = jz if jz < nz // 2 else jz - nz
            for kx in range(nx // 2):
                if jz == nz // 2:
                    continue
                d[(kx, kz)] = fh[jz, kx]
                if kx > 0:
                    d[(-kx, -kz)] = np.conj(fh[jz, kx])
        return d
    A, B = full(ah), full(bh)
    for jz in range(nz):
        kz = jz if jz < nz // 2 else jz - nz
        for kx in range(nx // 2 + 1):
            exact = 0j
            if jz != nz // 2 and kx != nx // 2:
                for (p, q), v in A.items():
                    w = B.get((kx - p, kz - q))
                    if w is not None:
                        exact += v * w
            assert abs(prod[jz, kx] - exact) < 1e-14


def test_parseval_on_padded_grid():
    rng = np.random.default_rng(3)
    nx, nz = 12, 16
    fh = _random_spec(rng, nx, nz)[0]
    f = to_phys(fh[None], nx, nz)[0]
    w = np.full(fh.shape, 2.0)
    w[:, 0] = 1.0
    assert abs(np.mean(f ** 2) - np.sum(w * np.abs(fh) ** 2)) < 1e-13


def test_mask_and_wavenumbers():
    k1, k3 = wavenumbers(8, 6, 2 * np.pi, 4 * np.pi)
    assert np.allclose(k1[0], [0, 1, 2, 3, 0]) and np.allclose(k3[:, 0], [0, 0.5, 1.0, 0, -1.0, -0.5])
    m = retained_mask(8, 6)
    assert not m[3].any() and not m[:, 4].any() and m.sum() == 5 * 4


@pytest.mark.parametrize("nx", [6])
def test_odd_half_rejected(nx):
    with pytest.raises(ValueError):
        padded_shape(7, 8)
