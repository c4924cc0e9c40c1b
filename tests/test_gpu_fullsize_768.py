"""GPU checks at 768 x 769 x 768 (physical 1152 x 769 x 1152), the largest workload, in FP64 and in the
double-float precision path.

At this size the full workspace would not leave room on the device, so lmvd_create picks the lean layout
by itself (memory_layout 0); its footprint is asserted below the device capacity. The outputs of the first
substage after a start-up are checked, as at 512 x 513 x 512, by properties that hold at any size (exact
discrete mass conservation of m^c in B-coefficient space, Sec. 4.2 with the exact D* of Appendix C;
Hermitian symmetry of the kx = 0 column; finite values), against the oracle's own matrices on sampled
modes (the m^c solve and the stage-n RK update are independent per (kx, kz)), and FP64 against
double-float. Device tensors are moved to the host one field at a time: the device holds the context.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

W = "rt768"


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


@pytest.fixture(scope="module")
def ops():
    from _pairs import oracle_config, workload
    from oracle.lmvd import Operators
    return Operators(oracle_config(workload(W)))


def _run(L, precision):
    import gc
    from _pairs import workload
    from paper_2206_09878_gb300.rt_inputs import rt_state
    gc.collect()
    torch.cuda.empty_cache()   # earlier tests' tensors, cached by torch, would not leave room for the context
    w = workload(W)
    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"],
                                n_startup=2, precision=precision)
    ctx = L.Context(cfg)
    out = {"device_bytes": L.lmvd_device_bytes(ctx.h)}
    st = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rt_state(**w).items()}
    ctx.set_state(st)
    del st
    torch.cuda.empty_cache()
    before = ctx.get_state()
    out["before"] = {k: v.cpu().numpy() for k, v in before.items()}
    del before
    torch.cuda.empty_cache()
    ctx.advance_substage()
    for name in ("RHO_T", "MC1", "MC2", "MC3", "R_OMEGA2", "R_PHI2"):
        out[name] = ctx.field(getattr(L, "LMVD_FIELD_" + name)).cpu().numpy()
        torch.cuda.empty_cache()
    after = ctx.get_state()
    out["after"] = {k: v.cpu().numpy() for k, v in after.items()}
    del after
    out["status"] = L.lmvd_status(ctx.h)
    ctx.close()
    torch.cuda.empty_cache()
    return out


@pytest.fixture(scope="module")
def run0(L):
    return _run(L, 0)


def _sample_modes(ops, n=12, seed=5):
    rng = np.random.default_rng(seed)
    idx = np.nonzero(ops.kmask.ravel())[0]
    return np.sort(rng.choice(idx, size=n, replace=False))


def test_footprint_fits_the_device(run0):
    total = torch.cuda.get_device_properties(0).total_memory
    print("device bytes %.1f GB of %.1f GB" % (run0["device_bytes"] / 1e9, total / 1e9))
    assert 0 < run0["device_bytes"] < total
    assert run0["status"] == 0


def test_mass_conservation_and_symmetry_768(run0, ops):
    D = ops.basis.D
    ds = np.array([D[i, i + 1] for i in range(D.shape[0])])
    rt, m1, m2, m3 = run0["RHO_T"], run0["MC1"], run0["MC2"], run0["MC3"]
    res = rt + 1j * ops.k1 * m1 + 1j * ops.k3 * m3 + ds[:, None, None] * (m2[1:] - m2[:-1])
    assert np.linalg.norm(res) < 1e-13 * np.linalg.norm(rt)
    after = run0["after"]
    for k, v in after.items():
        assert np.all(np.isfinite(v)), k
    nz = after["z"].shape[1]
    for k in ("z", "om", "m2"):
        col = after[k][:, :, 0]
        a = col[:, 1:nz // 2]
        b = np.conj(col[:, nz // 2 + 1:][:, ::-1])
        assert np.abs(a - b).max() <= 1e-13 * np.abs(col).max() + 1e-300, k


def test_mc_solve_and_update_on_sampled_modes_768(run0, ops):
    """The m^c solve and the stage-n Omega2 / m2^d updates of sampled modes with the oracle's matrices."""
    from oracle import banded
    from oracle.lmvd import _ax0
    sel = _sample_modes(ops)
    ny = ops.cfg.ny
    dt = ops.cfg.dt
    k2 = ops.k2.ravel()[sel]
    rt = run0["RHO_T"].reshape(ny, -1)[:, sel]
    rhs = np.zeros((ny + 1, len(sel)), complex)
    rhs[1:ny] = -(ops.Bs[1] @ rt)[1:ny]
    m2c = banded.solve_k2(ops.Amc2, ops.Amc0, k2, rhs, ops.Amc1)
    got = run0["MC2"].reshape(ny + 1, -1)[:, sel]
    assert np.linalg.norm(got - m2c) <= 1e-12 * np.linalg.norm(m2c)
    om0 = run0["before"]["om"].reshape(ny, -1)[:, sel]
    v = _ax0(ops.Bg[0], om0) + dt * 0.5 * run0["R_OMEGA2"].reshape(ny, -1)[:, sel]
    v[0] = 0
    v[ny - 1] = 0
    om1 = banded.solve(ops.A_interp, v)
    assert np.linalg.norm(run0["after"]["om"].reshape(ny, -1)[:, sel] - om1) <= 1e-12 * np.linalg.norm(om1)
    m20 = run0["before"]["m2"].reshape(ny + 1, -1)[:, sel]
    phi = _ax0(ops.Ss[2], m20) - k2 * _ax0(ops.Ss[0], m20)
    v = phi + dt * 0.5 * run0["R_PHI2"].reshape(ny + 1, -1)[:, sel]
    v[:2] = 0
    v[ny - 1:] = 0
    m21 = banded.solve_k2(ops.Amd2, ops.Amd0, k2, v, ops.Amd1)
    assert np.linalg.norm(run0["after"]["m2"].reshape(ny + 1, -1)[:, sel] - m21) <= 1e-12 * np.linalg.norm(m21)


def test_double_float_path_agrees_with_fp64_768(L, run0):
    r1 = _run(L, 1)
    for k in ("z", "om", "m2"):
        a0, a1 = run0["after"][k], r1["after"][k]
        rel = np.linalg.norm(a1 - a0) / np.linalg.norm(a0)
        assert rel < 1e-12, (k, rel)
