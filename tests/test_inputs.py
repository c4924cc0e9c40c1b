"""CPU checks of the seeded input recipe (paper_2206_09878_gb300/rt_inputs.py) that feeds the oracle and the
CUDA path alike: determinism, the spectral layout, the Nyquist and Hermitian conventions, the velocity band
and its wall rows, linearity in the velocity amplitude, the flat-interface case, and the torch form of the
eta -> z map used by the gradient configuration."""
import numpy as np
import pytest

from paper_2206_09878_gb300.rt_inputs import (PAPER_RT, WORKLOADS, eta_modes, rt_paper_state, rt_state,
                                              z_from_eta_torch)

SMALL = dict(WORKLOADS["rt32"], nx=16, ny=17, nz=12, kmax=3)


def _kz(nz):
    j = np.arange(nz)
    return np.where(j < nz // 2, j, j - nz)


def test_seeded_and_deterministic():
    a, b = rt_state(**SMALL), rt_state(**SMALL)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    c = rt_state(**dict(SMALL, seed=SMALL["seed"] + 1))
    assert not np.array_equal(a["z"], c["z"]) and not np.array_equal(a["om"], c["om"])


def test_layout_nyquist_and_hermitian_column():
    w = SMALL
    st = rt_state(**w)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    assert st["z"].shape == st["om"].shape == (ny, nz, nx // 2 + 1)
    assert st["m2"].shape == (ny + 1, nz, nx // 2 + 1)
    assert st["mm1"].shape == st["mm3"].shape == (ny,)
    for k in ("z", "om", "m2"):
        a = st[k]
        assert a.dtype == np.complex128
        assert not a[:, nz // 2, :].any() and not a[:, :, nx // 2].any(), k     # Nyquist slots
        col = a[:, :, 0]
        assert np.allclose(col[:, 1:nz // 2], np.conj(col[:, nz - 1:nz // 2:-1]), atol=1e-15), k
        assert np.allclose(col[:, 0].imag, 0.0, atol=1e-15), k


def test_velocity_band_and_wall_rows():
    w = SMALL
    st = rt_state(**w)
    nx, ny, nz, kmax = w["nx"], w["ny"], w["nz"], w["kmax"]
    kx = np.arange(nx // 2 + 1)[None, :]
    kz = _kz(nz)[:, None]
    band = (kx ** 2 + kz ** 2 > 0) & (kx ** 2 + kz ** 2 <= kmax ** 2)
    for k in ("om", "m2"):
        a = st[k]
        assert not a[:, ~band].any(), k                     # nothing outside the band
        assert np.count_nonzero(np.abs(a).sum(0)) == band.sum(), k   # every band mode is populated
    assert not st["m2"][[0, 1, ny - 1, ny]].any()           # m2^d = dm2^d/dy = 0 at the walls
    assert not st["om"][[0, ny - 1]].any()
    assert not st["mm1"].any() and not st["mm3"].any()


def test_linear_in_velocity_amplitude_and_z_independent_of_it():
    a = rt_state(**SMALL)
    b = rt_state(**dict(SMALL, u_rms=2 * SMALL["u_rms"]))
    assert np.allclose(b["om"], 2 * a["om"], rtol=1e-14, atol=0)
    assert np.allclose(b["m2"], 2 * a["m2"], rtol=1e-14, atol=0)
    assert np.array_equal(a["z"], b["z"])


def test_flat_interface_has_only_the_mean_mode_and_z_in_unit_interval():
    st = rt_state(**dict(SMALL, eta_rms=0.0))
    z = st["z"]
    rest = z.copy()
    rest[:, 0, 0] = 0
    assert np.abs(rest).max() < 1e-15
    prof = z[:, 0, 0].real                                  # the tanh profile in y: heavy (z = 1) on top
    assert np.all(np.diff(prof) >= -1e-15) and prof[0] < 0.01 and prof[-1] > 0.99
    zr = np.fft.irfft2(rt_state(**SMALL)["z"], s=(SMALL["nz"], SMALL["nx"]), axes=(1, 2), norm="forward")
    assert zr.min() > -0.05 and zr.max() < 1.05             # band-limited samples of a [0, 1] field


def test_torch_eta_map_equals_the_generator():
    torch = pytest.importorskip("torch")
    w = SMALL
    modes, theta, amp = eta_modes(**w)
    amps = torch.full((len(modes),), amp * w["eta_rms"], dtype=torch.float64)
    zt = z_from_eta_torch(amps, modes, theta, **w).numpy()
    z = rt_state(**w)["z"]
    assert np.abs(zt - z).max() <= 1e-15 * max(1.0, np.abs(z).max())


@pytest.mark.parametrize("name", sorted(PAPER_RT))
def test_paper_state_is_at_rest_with_z_in_unit_interval(name):
    w = dict(PAPER_RT[name])
    w.update(nx=16, nz=16, ny=min(w["ny"], 65))
    st = rt_paper_state(**w)
    assert not st["om"].any() and not st["m2"].any() and not st["mm1"].any() and not st["mm3"].any()
    zr = np.fft.irfft2(st["z"], s=(16, 16), axes=(1, 2), norm="forward")
    assert zr.min() > -0.05 and zr.max() < 1.05
    # h(x, z) = h(z, x): the sampled field is symmetric under x <-> z
    assert np.allclose(zr, np.transpose(zr, (0, 2, 1)), atol=1e-12)
