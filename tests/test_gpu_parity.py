"""GPU parity: the CUDA substage (through the C-ABI) against the FP64 oracle on the same seeded inputs.

Tolerance: relative L2 error <= 1e-12 per field for z, Omega2, m2^d and the whole m1, m3 momentum
components (the plane means are compared as part of their component: alone they are ~1e-6 of
the fluctuations and their relative error is amplified ~1e3 by cancellation, as the oracle shows
when its own input is perturbed by one rounding unit).

The intermediate fields of every substage are asserted too (tests/_pairs.py, intermediate_check):
* dz/dt against the oracle's within max(1e-12, 128 u |z| / (dt |dz/dt|)), the 1/dt round-off
  amplification of the BDF-like guess (Eq. dzdt_guesses, Sec. 3.3.1);
* R_z against the oracle's within 1e-12;
* rho_t, m^c and the three right-hand sides against the oracle's steps applied to the GPU's own
  dz/dt, within 8 times the spread a rounding model of the transforms and band evaluations gives
  (never below 1e-12).
Bounds are scaled by 2^-48 / 2^-53 = 32 for the double-float transforms and products.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2206_09878_gb300 import lmvd
    return lmvd


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,over", [
    ("rt32", {}),
    ("rt32", dict(nx=24, ny=21, nz=16, kmax=3)),
    ("rt32", dict(p=4, ny=25)),
    ("rt32", dict(memory_layout=2)),
    ("rt32", dict(nx=12, ny=11, nz=24, p=5, kmax=2)),    # 18-point x transforms: 6 elements per thread
    ("rt32", dict(nx=8, ny=10, nz=8, p=4, kmax=2)),      # 12-point transforms: one thread per transform
])
def test_substages_match_oracle(L, name, over, precision):
    """precision 0: FP64 throughout; 1: double-float transforms and products, FP64 spectral steps.
    memory_layout 2: the lean workspace (three product batches, 2-field transform intermediate)."""
    from _pairs import (compare_states, gpu_intermediates, intermediate_check, make_pair, oracle_intermediates,
                        to_numpy, to_torch)
    S, ctx, st, cfg = make_pair(L, name, precision=precision, **over)
    S.set_state(**st)
    ctx.set_state(to_torch(st))
    nsub = 2 * 5 if not over or "memory_layout" in over else 4
    worst = {}
    over_tol = []
    prev = st
    for s in range(nsub):
        S.advance_substage()
        ctx.advance_substage()
        gpu = to_numpy(ctx.get_state())
        ctx.synchronize()
        e = compare_states(S, gpu, S.state())
        fe, tol = intermediate_check(S, cfg, gpu_intermediates(L, ctx), oracle_intermediates(S), precision,
                                     state=prev)
        prev = gpu
        print("substage", s, {k: "%.1e" % v for k, v in {**e, **fe}.items()}, "tol %.1e" % tol["zdot"])
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
        over_tol += [(s, k, v, tol[k]) for k, v in fe.items() if not v <= tol[k]]
    ctx.close()
    assert all(v <= TOL for v in worst.values()), worst
    assert not over_tol, over_tol


@pytest.mark.parametrize("precision", [0, 1])
def test_constant_density_and_flat_interface(L, precision):
    """Degenerate cases: rho_h = rho_l (f' = 0, m^c = 0) and a state at rest with a flat interface."""
    from _pairs import compare_states, make_pair, to_numpy, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", precision=precision, ratio=1.0 + 1e-12, eta_rms=0.0, u_rms=0.0)
    S.set_state(**st)
    ctx.set_state(to_torch(st))
    for _ in range(2):
        S.advance_substage()
        ctx.advance_substage()
    gpu = to_numpy(ctx.get_state())
    e = compare_states(S, gpu, S.state())
    assert e["z"] <= TOL
    assert np.abs(gpu["om"]).max() == 0.0 and np.abs(gpu["m2"]).max() == 0.0
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_restart_from_history_is_bitwise(L, precision):
    """get_state(history) -> set_state(history) resumes the same sequence bit for bit."""
    from _pairs import make_pair, to_numpy, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", precision=precision)
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    hist = ctx.history_buffer()
    mid = ctx.get_state(history=hist)
    ctx.advance_substage()
    ctx.advance_substage()
    a = to_numpy(ctx.get_state())
    ctx.set_state(mid, history=hist)
    ctx.advance_substage()
    ctx.advance_substage()
    b = to_numpy(ctx.get_state())
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    ctx.close()


def test_host_buffers_equal_device_buffers(L):
    from _pairs import make_pair, to_numpy, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32")
    ctx.set_state(to_torch(st, "cpu"))
    ctx.advance_substage()
    host = ctx.get_state(ctx.empty_state("cpu", pin=True))
    ctx.synchronize()
    dev = to_numpy(ctx.get_state())
    for k in host:
        assert np.array_equal(host[k].numpy(), dev[k]), k
    ctx.close()
