"""GPU: the index-checked build (liblmvd_check.so, -DLMVD_CHECK) on odd and ragged sizes.

compute-sanitizer is closed on this machine, so memory safety is checked by the library itself: in the
checked build every checked access tests its index against the extent of its array first, skips the
access if it is outside and sets a device word that lmvd_synchronize turns into LMVD_ERR_OUT_OF_BOUNDS
(nothing traps). Here that build runs, in a child process of its own (LMVD_LIBRARY selects it), the
odd-structured parity grids (24 x 21 x 16, 12 x 11 x 24 with spline order 5 and 18-point transforms,
8 x 10 x 8 with order 4 and 12-point transforms) in both precisions and both memory layouts, with
CUDA-graph replay, one adjoint substage and the transforms of the C-ABI; every status must stay clear
and the states must still match the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_CHECK = os.path.join(ROOT, "paper_2206_09878_gb300", "liblmvd_check.so")

SCRIPT = r"""
import sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
import numpy as np
import torch
from paper_2206_09878_gb300 import lmvd as L
from _pairs import compare_states, make_pair, to_numpy, to_torch
assert L.lmvd_checked_build() == 1
cases = [dict(nx=24, ny=21, nz=16, kmax=3), dict(nx=12, ny=11, nz=24, p=5, kmax=2),
         dict(nx=8, ny=10, nz=8, p=4, kmax=2)]
for over in cases:
    for precision, layout in ((0, 1), (1, 2), (0, 2), (1, 1)):
        S, ctx, st, cfg = make_pair(L, "rt32", precision=precision, memory_layout=layout, **over)
        S.set_state(**st)
        ctx.set_state(to_torch(st))
        for s in range(4):
            S.advance_substage()
            ctx.advance_substage()
        code = L._lib.lmvd_synchronize(ctx.h)
        assert code == 0, (over, precision, layout, code)
        e = compare_states(S, to_numpy(ctx.get_state()), S.state())
        assert max(e.values()) <= 1e-12, (over, precision, layout, e)
        ctx.close()
    # graph replay on a side stream (captured substages), then one adjoint substage (FP64)
    side = torch.cuda.Stream()
    S, ctx, st, cfg = make_pair(L, "rt32", **over)
    with torch.cuda.stream(side):
        ctx2 = L.Context(ctx.cfg, stream=side)
        ctx2.set_state(to_torch(st))
        for s in range(12):
            ctx2.advance_substage()
        assert L._lib.lmvd_synchronize(ctx2.h) == 0
        ctx2.close()
    ctx.set_state(to_torch(st))
    nb = L.lmvd_state_bytes(ctx.h)
    hb = L.lmvd_history_bytes(ctx.h)
    g = torch.Generator(device="cuda").manual_seed(3)
    sbar = torch.randn(nb // 8, dtype=torch.float64, device="cuda", generator=g)
    hbar = torch.zeros(hb // 8, dtype=torch.float64, device="cuda")
    sout = torch.zeros(nb // 8, dtype=torch.float64, device="cuda")
    hout = torch.zeros(hb // 8, dtype=torch.float64, device="cuda")
    L.lmvd_adjoint_substage(ctx.h, sbar, hbar, sout, hout)
    assert L._lib.lmvd_synchronize(ctx.h) == 0
    # the transforms of the C-ABI and the allocation-free one
    nf = 2
    spec = torch.zeros((nf, cfg.ny, cfg.nz, cfg.nx // 2 + 1), dtype=torch.complex128, device="cuda")
    spec.real.normal_(generator=g)
    phys = torch.zeros((nf, cfg.ny, 3 * cfg.nz // 2, 3 * cfg.nx // 2), dtype=torch.float64, device="cuda")
    L.lmvd_inverse_transform(ctx.h, spec, phys, nf)
    L.lmvd_forward_transform(ctx.h, phys, spec, nf)
    L.lmvd_inverse_transform_noalloc(cfg.nx, cfg.ny, cfg.nz, spec, phys, nf)
    assert L._lib.lmvd_synchronize(ctx.h) == 0
    ctx.close()
print("CHECKED BUILD OK")
"""


def test_checked_build_runs_odd_sizes_in_bounds():
    assert os.path.exists(LIB_CHECK), "liblmvd_check.so is built by build()"
    env = dict(os.environ, LMVD_LIBRARY=LIB_CHECK)
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT, "tests": HERE}], env=env,
                       capture_output=True, text=True, timeout=1200)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0 and "CHECKED BUILD OK" in r.stdout
