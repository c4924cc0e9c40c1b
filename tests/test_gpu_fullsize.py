"""GPU checks at the full workloads 512 x 513 x 512 (the configuration bench.py times) and 256 x 257 x 256
(density ratio 25.7), including 20 RK steps at 256 x 257 x 256.

The oracle cannot run this grid in test time, so the GPU outputs are checked
* by properties that hold at any size: exact discrete mass conservation of m^c in B-coefficient space
  (Sec. 4.2, Eq. COM_fourier with the exact D* of Appendix C), Hermitian symmetry of the kx = 0 column,
  finite values;
* against the oracle one mode at a time on sampled modes: the m^c solve (Eq. COM_fourier, CF_fourier,
  mc_recon) and the RK2 update with its wall rows are independent per (kx, kz), so the oracle's own
  matrices solve them for a handful of modes from the GPU's inputs;
* against each other: the FP64 and the double-float transform paths after the same substages.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


@pytest.fixture(scope="module", params=["rt512", "rt256"])
def W(request):
    return request.param


@pytest.fixture(scope="module")
def ops(W):
    from _pairs import oracle_config, workload
    from oracle.lmvd import Operators
    return Operators(oracle_config(workload(W)))


def _run(L, W, precision, nsub, history=False):
    import gc
    from _pairs import workload
    from paper_2206_09878_gb300.rt_inputs import rt_state
    gc.collect()
    torch.cuda.empty_cache()
    w = workload(W)
    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"],
                                n_startup=4, precision=precision)
    ctx = L.Context(cfg)
    st = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rt_state(**w).items()}
    ctx.set_state(st)
    for _ in range(nsub - 1):
        ctx.advance_substage()
    hist = ctx.history_buffer()
    before = {k: v.clone() for k, v in ctx.get_state(history=hist).items()}
    if history:
        before["history"] = hist.cpu().numpy()
    del hist
    ctx.advance_substage()
    fields = {name: ctx.field(getattr(L, "LMVD_FIELD_" + name)) for name in
              ("RHO_T", "MC1", "MC2", "MC3", "ZDOT", "R_OMEGA2", "R_PHI2", "R_MEANS")}
    after = ctx.get_state()
    ctx.synchronize()
    ctx.close()
    return before, fields, after


@pytest.fixture(scope="module")
def run0(L, W):
    return _run(L, W, 0, 2)


def _sample_modes(ops, n=12, seed=5):
    rng = np.random.default_rng(seed)
    idx = np.nonzero(ops.kmask.ravel())[0]
    return np.sort(rng.choice(idx, size=n, replace=False))


def test_mass_conservation_and_symmetry_full_size(run0, ops):
    before, f, after = run0
    k1 = torch.from_numpy(ops.k1).cuda()
    k3 = torch.from_numpy(ops.k3).cuda()
    D = ops.basis.D
    ds = torch.from_numpy(np.array([D[i, i + 1] for i in range(D.shape[0])])).cuda()
    rt, m1, m2, m3 = f["RHO_T"], f["MC1"], f["MC2"], f["MC3"]
    dm2 = ds[:, None, None] * (m2[1:] - m2[:-1])
    res = rt + 1j * k1 * m1 + 1j * k3 * m3 + dm2
    rel = float(torch.linalg.vector_norm(res) / torch.linalg.vector_norm(rt))
    assert rel < 1e-13, rel
    for k, v in after.items():
        assert bool(torch.isfinite(torch.view_as_real(v) if v.is_complex() else v).all()), k
    nz = after["z"].shape[1]
    for k in ("z", "om", "m2"):
        col = after[k][:, :, 0]
        a = col[:, 1:nz // 2]
        b = torch.flip(col[:, nz // 2 + 1:], dims=[1]).conj()
        # the forward transforms produce kz and -kz along different butterfly paths: conjugate to rounding
        assert float((a - b).abs().max()) <= 1e-13 * float(col.abs().max()) + 1e-300, k


def test_mc_solve_on_sampled_modes_matches_oracle(run0, ops):
    from oracle import banded
    from oracle.lmvd import _ax0
    _, f, _ = run0
    sel = _sample_modes(ops)
    ny = ops.cfg.ny
    rt = f["RHO_T"].reshape(ny, -1)[:, sel].cpu().numpy()
    rhs = np.zeros((ny + 1, len(sel)), complex)
    rhs[1:ny] = -(ops.Bs[1] @ rt)[1:ny]
    k2 = ops.k2.ravel()[sel]
    m2 = banded.solve_k2(ops.Amc2, ops.Amc0, k2, rhs)
    got = f["MC2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got - m2) <= 1e-12 * np.linalg.norm(m2)
    k = np.sqrt(k2)
    mpar = 1j * (rt + _ax0(ops.D, m2)) / k
    m1 = ops.k1.ravel()[sel] / k * mpar
    got1 = f["MC1"].reshape(ny, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got1 - m1) <= 1e-12 * max(np.linalg.norm(m1), 1e-300)


def test_wall_rows_hold_full_size(run0, ops):
    """No-slip rows of the update: m2^d(+-1) = dm2^d/dy(+-1) = 0 and Omega2(+-1) = 0 on sampled modes."""
    _, _, after = run0
    sel = _sample_modes(ops, seed=9)
    ny = ops.cfg.ny
    m2 = after["m2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    om = after["om"].reshape(ny, -1)[:, sel].cpu().numpy()
    scale2, scale1 = np.abs(m2).max(), np.abs(om).max()
    assert np.abs(m2[[0, ny]]).max() <= 1e-14 * scale2
    dm = ops.basis.Ss[1][[0, ny]] @ m2
    assert np.abs(dm).max() <= 1e-12 * scale2 * ny
    assert np.abs(om[[0, ny - 1]]).max() <= 1e-14 * scale1


@pytest.mark.parametrize("precision", [0, 1])
def test_stage_n_update_on_sampled_modes_matches_oracle(L, W, ops, precision):
    """First substage after start-up (stage n, al = 1/2, be = 0): rebuild the Omega2 and m2^d updates of
    sampled modes with the oracle's matrices from the GPU's state and RHS (FP64 and double-float)."""
    from oracle import banded
    from oracle.lmvd import _ax0
    before, f, after = _run(L, W, precision, 1)
    sel = _sample_modes(ops, seed=11)
    ny = ops.cfg.ny
    dt = ops.cfg.dt
    om0 = before["om"].reshape(ny, -1)[:, sel].cpu().numpy()
    rom = f["R_OMEGA2"].reshape(ny, -1)[:, sel].cpu().numpy()
    v = _ax0(ops.Bg[0], om0) + dt * 0.5 * rom
    v[0] = 0
    v[ny - 1] = 0
    om1 = banded.solve(ops.A_interp, v)
    got = after["om"].reshape(ny, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got - om1) <= 1e-12 * np.linalg.norm(om1)
    m20 = before["m2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    rphi = f["R_PHI2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    k2 = ops.k2.ravel()[sel]
    phi = _ax0(ops.Ss[2], m20) - k2 * _ax0(ops.Ss[0], m20)
    v = phi + dt * 0.5 * rphi
    v[:2] = 0
    v[ny - 1:] = 0
    m21 = banded.solve_k2(ops.Amd2, ops.Amd0, k2, v)
    got = after["m2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got - m21) <= 1e-12 * np.linalg.norm(m21)


def test_double_float_path_agrees_with_fp64_full_size(L, W, run0):
    _, f0, a0 = run0
    _, f1, a1 = _run(L, W, 1, 2)
    for k in ("z", "om", "m2"):
        rel = float(torch.linalg.vector_norm(a1[k] - a0[k]) / torch.linalg.vector_norm(a0[k]))
        assert rel < 1e-12, (k, rel)


@pytest.mark.parametrize("W", ["rt256"], indirect=True)
def test_twenty_rk_steps_256(L, ops, W):
    """20 RK steps (40 substages) at 256 x 257 x 256, dt = 2e-4, density ratio 25.7: the state stays finite
    and Hermitian, m^c of the last substage conserves mass exactly, and the last substage (stage ', al = 1,
    be = -1/2) updates Omega2 and m2^d of sampled modes as the oracle's matrices do from the GPU's state,
    RHS and previous RHS (from the history)."""
    from oracle import banded
    from oracle.lmvd import _ax0
    before, f, after = _run(L, W, 0, 40, history=True)
    for k, v in after.items():
        assert bool(torch.isfinite(torch.view_as_real(v) if v.is_complex() else v).all()), k
    D = ops.basis.D
    ds = torch.from_numpy(np.array([D[i, i + 1] for i in range(D.shape[0])])).cuda()
    k1 = torch.from_numpy(ops.k1).cuda()
    k3 = torch.from_numpy(ops.k3).cuda()
    res = f["RHO_T"] + 1j * k1 * f["MC1"] + 1j * k3 * f["MC3"] + ds[:, None, None] * (f["MC2"][1:] - f["MC2"][:-1])
    assert float(torch.linalg.vector_norm(res) / torch.linalg.vector_norm(f["RHO_T"])) < 1e-13
    ny, nz, nxh = ops.cfg.ny, ops.cfg.nz, ops.cfg.nx // 2 + 1
    M = nz * nxh
    S, Sp = 16 * ny * M, 16 * (ny + 1) * M
    h = before["history"]
    # history blob: 16-byte header, z^{s-1}, z^{s-2}, z^{s-3}, dz/dt^{s-1}, RHS_Omega2, RHS_phi2, means
    r_om_prev = h[16 + 4 * S:16 + 5 * S].view(np.complex128).reshape(ny, -1)
    r_phi_prev = h[16 + 5 * S:16 + 5 * S + Sp].view(np.complex128).reshape(ny + 1, -1)
    sel = _sample_modes(ops, seed=13)
    dt = ops.cfg.dt
    om0 = before["om"].reshape(ny, -1)[:, sel].cpu().numpy()
    v = _ax0(ops.Bg[0], om0) + dt * (f["R_OMEGA2"].reshape(ny, -1)[:, sel].cpu().numpy() - 0.5 * r_om_prev[:, sel])
    v[0] = 0
    v[ny - 1] = 0
    om1 = banded.solve(ops.A_interp, v)
    got = after["om"].reshape(ny, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got - om1) <= 1e-12 * np.linalg.norm(om1)
    m20 = before["m2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    k2 = ops.k2.ravel()[sel]
    phi = _ax0(ops.Ss[2], m20) - k2 * _ax0(ops.Ss[0], m20)
    v = phi + dt * (f["R_PHI2"].reshape(ny + 1, -1)[:, sel].cpu().numpy() - 0.5 * r_phi_prev[:, sel])
    v[:2] = 0
    v[ny - 1:] = 0
    m21 = banded.solve_k2(ops.Amd2, ops.Amd0, k2, v)
    got = after["m2"].reshape(ny + 1, -1)[:, sel].cpu().numpy()
    assert np.linalg.norm(got - m21) <= 1e-12 * np.linalg.norm(m21)
