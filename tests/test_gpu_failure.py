"""GPU: failure detection and diagnostics, without faulting the GPU.

* A non-finite value injected on the host into the state given to lmvd_set_state (nan in z, inf in Omega2)
  propagates through a substage; the device check marks it and lmvd_synchronize returns
  LMVD_ERR_NONFINITE (latched in lmvd_status). A clean run returns LMVD_OK.
* The diagnostics record (lmvd_diagnostics) matches the oracle: the relative change of each fixed-point
  application |dz/dt^{k+1} - dz/dt^k| / |dz/dt^{k+1}| is the oracle's fp_residuals (Sec. 3.1), and the
  relative mass residual of m^c is at rounding level (Sec. 4.2, exact D*).
* The record's kinetic energy, max |m| and bottom value of <m2^c> match the same quantities formed from the
  oracle's fields, and take their closed-form values for a uniform stream (KE = U^2 / 2 times the volume).
* At density ratio 100 with a sharp interface the fixed point does not converge (the oracle shows
  relative changes above 1 throughout); lmvd_synchronize returns LMVD_ERR_FP_DIVERGED. At the paper's
  density ratios it stays clean.
* The transforms' tile copies wait on an mbarrier with a time limit: a copy that cannot complete (more
  bytes expected than sent, through lmvd_tile_wait_probe) makes the CTA give up after ~1 s and set the
  status bit that lmvd_synchronize reports as LMVD_ERR_CUDA, with no fault and the device still usable.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NONFINITE, FP_DIVERGED = -4, -6


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


@pytest.mark.parametrize("field,value", [("z", np.nan), ("om", np.inf)])
def test_nonfinite_state_is_detected(L, field, value):
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32")
    st = {k: v.copy() for k, v in st.items()}
    st[field][cfg.ny // 2, 1, 1] = value
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    assert L._lib.lmvd_synchronize(ctx.h) == NONFINITE
    assert L.lmvd_status(ctx.h) == NONFINITE
    ctx.close()


def test_clean_run_reports_ok(L):
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32")
    L.lmvd_diagnostics_enable(ctx.h, True)
    ctx.set_state(to_torch(st))
    for _ in range(4):
        ctx.advance_substage()
    assert L._lib.lmvd_synchronize(ctx.h) == 0
    ctx.close()


def test_diagnostics_match_oracle(L):
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32")
    L.lmvd_diagnostics_enable(ctx.h, True)
    S.set_state(**st)
    ctx.set_state(to_torch(st))
    for s in range(3):
        S.advance_substage()
        ctx.advance_substage()
        d = L.lmvd_diagnostics(ctx.h)
        print(s, d, S.fp_residuals)
        assert d["substage"] == s
        assert d["mass_residual"] < 1e-13
        assert len(d["fp_changes"]) == cfg.kf
        for g, o in zip(d["fp_changes"], S.fp_residuals):
            assert abs(g - o) <= 1e-3 * o + 1e-11, (g, o)
    ctx.close()


def _oracle_energy(S):
    """(1/2) integral of |m^d + m^c|^2 / rho dV and max |m| from the oracle's fields of its last substage."""
    from oracle.lmvd import _ax0
    op, cfg = S.op, S.cfg
    m1c, m2c, m3c = S.trace["mc"]
    mcp = (op.phys(_ax0(op.Bg[0], m1c)), op.phys(_ax0(op.Sg0, m2c)), op.phys(_ax0(op.Bg[0], m3c)))
    m2 = sum((S.md_phys[i] + mcp[i]) ** 2 for i in range(3))
    b = op.basis
    integral = (b.t[cfg.p:cfg.p + cfg.ny] - b.t[:cfg.ny]) / cfg.p          # integral of each B_j
    wq = np.linalg.solve(b.Bg[0].T, integral)                             # weights at the Greville points
    plane = np.mean(0.5 * m2 / S.rho, axis=(1, 2))
    return cfg.lx * cfg.lz * float(wq @ plane), float(np.sqrt(m2.max()))


@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_energy_and_wall_flux_match_oracle(L, precision):
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", precision=precision)
    L.lmvd_diagnostics_enable(ctx.h, True)
    S.set_state(**st)
    ctx.set_state(to_torch(st))
    for s in range(3):
        S.advance_substage()
        ctx.advance_substage()
        d = L.lmvd_diagnostics(ctx.h)
        ke, mmax = _oracle_energy(S)
        mc2 = S.trace["mc"][1][0, 0, 0].real
        print(s, d["kinetic_energy"], ke, d["max_momentum"], mmax, d["mean_m2c_y0"], mc2)
        assert abs(d["kinetic_energy"] - ke) <= 1e-10 * ke
        assert abs(d["max_momentum"] - mmax) <= 1e-10 * mmax
        assert abs(d["mean_m2c_y0"] - mc2) <= 1e-9 * abs(mc2) + 1e-20
    ctx.close()


def test_diagnostics_uniform_stream_closed_form(L):
    """Uniform density, <m1> = U, <m3> = W (potential matching: Neumann rows keep them): KE = (U^2 + W^2)/2
    times lx lz (y1 - y0), max |m| = sqrt(U^2 + W^2), no mass flux (to rounding)."""
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", bc="potential")
    st = {k: np.zeros_like(v) for k, v in st.items()}
    st["z"][:, 0, 0] = 1.0                     # z = 1 everywhere: rho = rho_h = 1 exactly (Sec. 5 EOS)
    U, W = 0.3, -0.2
    st["mm1"][:] = U
    st["mm3"][:] = W
    L.lmvd_diagnostics_enable(ctx.h, True)
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    d = L.lmvd_diagnostics(ctx.h)
    vol = cfg.lx * cfg.lz * (cfg.y1 - cfg.y0)
    assert abs(d["kinetic_energy"] - 0.5 * (U * U + W * W) * vol) <= 1e-13 * vol
    assert abs(d["max_momentum"] - np.hypot(U, W)) <= 1e-14
    assert abs(d["mean_m2c_y0"]) <= 1e-14      # z is 1 up to the rounding of the spline sum
    ctx.close()


def test_fp_divergence_is_detected(L):
    """Density ratio 100, interface width 0.02 (beyond the paper's range): the iteration does not converge."""
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", ratio=100.0, width=0.02, n_startup=4)
    L.lmvd_diagnostics_enable(ctx.h, True)
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    d = L.lmvd_diagnostics(ctx.h)
    print(d)
    assert d["fp_changes"][-1] >= 0.5
    assert L._lib.lmvd_synchronize(ctx.h) == FP_DIVERGED
    ctx.close()


def test_oversized_grid_reports_oom_and_the_device_stays_usable(L):
    """1024 x 1025 x 1024 needs ~575 GB of workspace even in the lean layout: lmvd_create allocates the
    per-mode factors, fails the workspace allocation (a plain cudaMalloc error, no fault), releases what it
    holds and returns LMVD_ERR_OOM; a context created afterwards runs a clean substage."""
    import ctypes
    import gc
    from _pairs import make_pair, to_torch
    gc.collect()
    torch.cuda.empty_cache()
    cfg = L.lmvd_default_config(1024, 1025, 1024)
    h = ctypes.c_void_p()
    assert L._lib.lmvd_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -3     # LMVD_ERR_OOM
    assert not h.value
    S, ctx, st, _ = make_pair(L, "rt32")
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    assert L._lib.lmvd_synchronize(ctx.h) == 0
    ctx.close()


def test_tile_copy_wait_gives_up_and_is_reported(L):
    """The transforms' tile copies complete on an mbarrier that every thread waits for with a time limit
    (~1 s of SM clock). lmvd_tile_wait_probe runs that wait alone: with the expected bytes delivered it
    completes at once and the data arrive; with 16 bytes more expected than copied it can never complete,
    the CTA gives up after the limit and sets bit 2 of the status word (the bit lmvd_synchronize turns into
    LMVD_ERR_CUDA), and the device stays usable."""
    import time
    src = torch.arange(16, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.lmvd_tile_wait_probe(src, 0, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    t0 = time.time()
    L.lmvd_tile_wait_probe(src, 16, status)
    torch.cuda.synchronize()
    waited = time.time() - t0
    assert int(status.item()) == 4
    assert 0.2 < waited < 30
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32")
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    assert L._lib.lmvd_synchronize(ctx.h) == 0
    ctx.close()
