"""CPU checks of the host-side logic of the Goncharov validation (paper_2206_09878_gb300/rt_validation.py):
the line probes find the z = 1/2 crossing of the paper's initial interface (Sec. 5: h = 0.05 (cos 2 pi x +
cos 2 pi z) in 3D, so +-0.1 on the bubble and spike lines), the plateau finder recovers a known constant
velocity from a synthetic height record, and the 2D and 3D potential-flow velocities differ by the paper's
C = 3 against C = 1."""
import math

import numpy as np
import pytest

from paper_2206_09878_gb300.rt_validation import LineProbe, goncharov, initial_state, plateau


def _interface(nx, nz, dim, delta):
    x = np.arange(nx) / nx
    zc = np.arange(nz) / nz
    if dim == 3:
        return 0.05 * (np.cos(2 * np.pi * x)[None, :] + np.cos(2 * np.pi * zc)[:, None]) + delta
    return 0.1 * np.cos(2 * np.pi * x)[None, :] * np.ones((nz, 1)) + delta


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("delta", [0.0, 0.5])
def test_line_probes_find_the_interface(dim, delta):
    """z interpolated exactly at the Greville points (scipy's design matrix, independent of the library):
    the probes return the interface heights of the bubble and spike lines."""
    from scipy.interpolate import BSpline
    nx, ny, y0, y1, eps = 16, 257, -2.0, 2.0, 0.05
    nz = nx if dim == 3 else 4
    probe = LineProbe(nx, ny, nz, y0, y1, dim)
    t, k = probe.t, probe.k
    g = np.array([t[i + 1:i + k + 1].mean() for i in range(ny)])
    B = BSpline.design_matrix(g, t, k).toarray()
    h = _interface(nx, nz, dim, delta)
    zg = 0.5 * (1 + np.tanh((g[:, None, None] - h[None]) / (2 * eps)))
    coef = np.linalg.solve(B, zg.reshape(ny, -1)).reshape(zg.shape)
    zhat = np.fft.rfft2(coef, axes=(1, 2), norm="forward")
    zhat[:, nz // 2] = 0
    zhat[:, :, nx // 2] = 0
    hb, hs = probe.heights(zhat)
    assert abs(hb - (0.1 + delta)) < 2e-4, hb
    assert abs(hs - (-0.1 + delta)) < 2e-4, hs


@pytest.mark.parametrize("delta", [0.0, 0.5])
def test_initial_state_interface_within_one_knot_spacing(delta):
    """initial_state writes samples at uniform anchors as coefficients (a quasi-interpolant, like the input
    generator): the interface it represents sits within one knot spacing of the paper's h."""
    nx, ny, y0, y1 = 16, 257, -2.0, 2.0
    st = initial_state(nx, ny, nx, y0, y1, 3, delta)
    hb, hs = LineProbe(nx, ny, nx, y0, y1, 3).heights(st["z"])
    spacing = (y1 - y0) / (ny - 6 + 1)
    assert abs(hb - (0.1 + delta)) < spacing and abs(hs - (-0.1 + delta)) < spacing


def test_plateau_recovers_a_constant_velocity():
    t = np.linspace(0.0, 5.0, 2001)
    v = np.where(t < 3.0, 0.3 * np.tanh(3.0 * t), 0.3 + 0.2 * (t - 3.0) ** 2)   # accelerate, plateau, re-accelerate
    hb = np.concatenate([[0.0], np.cumsum(0.5 * (v[1:] + v[:-1]) * np.diff(t))])
    mean, spread, a, b = plateau(t, hb)
    assert abs(mean - 0.3) < 0.01 * 0.3, mean
    assert spread < 0.02 and b - a == pytest.approx(1.0, abs=0.01) and b <= 3.2


def test_plateau_without_a_plateau_is_nan():
    t = np.linspace(0.0, 0.5, 50)                        # shorter than the one-unit window
    assert all(math.isnan(x) for x in plateau(t, t ** 2))


def test_two_and_three_dimensional_potential_velocity():
    for at in (0.33, 0.5, 0.8):
        assert goncharov(at, 2) / goncharov(at, 3) == pytest.approx(1.0 / math.sqrt(3.0), rel=1e-14)
        # v^2 scales as At / (1 + At) at fixed wavenumber
        assert goncharov(at, 3) ** 2 / goncharov(0.5, 3) ** 2 == pytest.approx((at / (1 + at)) / (0.5 / 1.5))
