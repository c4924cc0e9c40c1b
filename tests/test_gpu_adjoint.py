"""GPU: the adjoint of one substage (lmvd_adjoint_substage) is the transpose of its Jacobian.

For x = (state, history) and a random output weight ybar, <ybar, J dx> must equal <J^T ybar, dx>.
J dx is measured by central differences, both of the CUDA forward substage and of the FP64 oracle's
substage (Algorithm 2 in oracle/lmvd.py) on 16 seeded directions; J^T ybar comes from the adjoint.
Perturbations are relative to each field's size, so a step h = 1e-6 keeps the truncation error of the
difference quotient below 1e-11 and its rounding error near 1e-10 of the products compared.
"""
import zlib

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def _layout(cfg):
    ny, nz, nxh = cfg.ny, cfg.nz, cfg.nx // 2 + 1
    S, Sp = (ny, nz, nxh), (ny + 1, nz, nxh)
    state = [("z", S, complex), ("om", S, complex), ("m2", Sp, complex), ("mm1", (ny,), float), ("mm3", (ny,), float)]
    hist = [("z1", S, complex), ("z2", S, complex), ("z3", S, complex), ("zdot", S, complex), ("r_om", S, complex),
            ("r_phi", Sp, complex), ("r_m", (2 * ny,), float)]
    return state, hist


def pack(cfg, d, which):
    state, hist = _layout(cfg)
    parts = []
    if which == "hist":
        parts.append(np.zeros(2, np.int64).view(np.uint8))
    for name, shape, kind in (state if which == "state" else hist):
        a = np.ascontiguousarray(np.asarray(d[name], dtype=np.complex128 if kind is complex else np.float64))
        assert a.shape == shape, (name, a.shape, shape)
        parts.append(a.reshape(-1).view(np.uint8))
    return np.concatenate(parts)


def unpack(cfg, blob, which):
    state, hist = _layout(cfg)
    off = 16 if which == "hist" else 0
    out = {}
    for name, shape, kind in (state if which == "state" else hist):
        dt = np.complex128 if kind is complex else np.float64
        nbytes = int(np.prod(shape)) * np.dtype(dt).itemsize
        out[name] = blob[off:off + nbytes].view(dt).reshape(shape).copy()
        off += nbytes
    return out


def dot(a, b):
    return sum(float(np.sum((np.conj(a[k]) * b[k]).real)) for k in a)


def _mask(cfg, d, state):
    """Zero the Nyquist slots (and the k = 0 slot of Omega2, m2^d) the method never reads."""
    nz, nx = cfg.nz, cfg.nx
    for k, v in d.items():
        if v.ndim == 3:
            v[:, nz // 2, :] = 0
            v[:, :, nx // 2] = 0
            if state and k in ("om", "m2"):
                v[:, 0, 0] = 0
    return d


def _random_like(rng, cfg, ref, state):
    out = {}
    for k, v in ref.items():
        scale = np.sqrt(np.mean(np.abs(v) ** 2)) if np.any(v) else 1.0
        if np.iscomplexobj(v):
            out[k] = scale * (rng.normal(size=v.shape) + 1j * rng.normal(size=v.shape))
        else:
            out[k] = scale * rng.normal(size=v.shape)
    return _mask(cfg, out, state)


def _gpu_map(L, ctx, cfg, st, hi):
    """One substage of the CUDA path from (state, history) -> (state', history') as numpy dicts."""
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
    hb = torch.from_numpy(pack(cfg, hi, "hist")).cuda()
    hb[:8] = torch.from_numpy(np.array([1], np.int64).view(np.uint8)).cuda()   # stage ' (odd substage)
    ctx.set_state(dev, history=hb)
    ctx.advance_substage()
    hout = ctx.history_buffer()
    so = ctx.get_state(history=hout)
    ctx.synchronize()
    return {k: v.cpu().numpy() for k, v in so.items()}, unpack(cfg, hout.cpu().numpy(), "hist")


@pytest.fixture(scope="module", params=["walls", "potential"])
def base(L, request):
    """A state and history after start-up and one substage of rt32 (32 x 33 x 32), at stage ', with
    no-slip walls or the potential-matching boundary rows."""
    from _pairs import make_pair, to_torch
    S, ctx, st, cfg = make_pair(L, "rt32", u_rms=1e-2, bc=request.param)
    ctx.set_state(to_torch(st))
    ctx.advance_substage()
    hb = ctx.history_buffer()
    so = ctx.get_state(history=hb)
    ctx.synchronize()
    x_state = {k: v.cpu().numpy() for k, v in so.items()}
    x_hist = unpack(cfg, hb.cpu().numpy(), "hist")
    return S, ctx, cfg, x_state, x_hist


def _adjoint(L, ctx, cfg, x_state, x_hist, yb_state, yb_hist):
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in x_state.items()}
    hb = torch.from_numpy(pack(cfg, x_hist, "hist")).cuda()
    hb[:8] = torch.from_numpy(np.array([1], np.int64).view(np.uint8)).cuda()
    ctx.set_state(dev, history=hb)
    nb = L.lmvd_state_bytes(ctx.h)
    sbi = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    hbi = torch.zeros(L.lmvd_history_bytes(ctx.h), dtype=torch.uint8, device="cuda")
    sbo = torch.from_numpy(pack(cfg, yb_state, "state")).cuda()
    hbo = torch.from_numpy(pack(cfg, yb_hist, "hist")).cuda()
    L.lmvd_adjoint_substage(ctx.h, sbo, hbo, sbi, hbi)
    return unpack(cfg, sbi.cpu().numpy(), "state"), unpack(cfg, hbi.cpu().numpy(), "hist")


@pytest.mark.parametrize("group", ["all", "state", "history"])
def test_adjoint_matches_gpu_central_differences(L, base, group):
    S, ctx, cfg, xs, xh = base
    rng = np.random.default_rng({"all": 1, "state": 2, "history": 3}[group])
    ys, yh = _gpu_map(L, ctx, cfg, xs, xh)
    ybs, ybh = _random_like(rng, cfg, ys, True), _random_like(rng, cfg, yh, False)
    dxs, dxh = _random_like(rng, cfg, xs, True), _random_like(rng, cfg, xh, False)
    if group == "state":
        dxh = {k: 0 * v for k, v in dxh.items()}
    if group == "history":
        dxs = {k: 0 * v for k, v in dxs.items()}
    xbs, xbh = _adjoint(L, ctx, cfg, xs, xh, ybs, ybh)
    h = 1e-6
    pp = _gpu_map(L, ctx, cfg, {k: xs[k] + h * dxs[k] for k in xs}, {k: xh[k] + h * dxh[k] for k in xh})
    mm = _gpu_map(L, ctx, cfg, {k: xs[k] - h * dxs[k] for k in xs}, {k: xh[k] - h * dxh[k] for k in xh})
    jvp_s = {k: (pp[0][k] - mm[0][k]) / (2 * h) for k in xs}
    jvp_h = {k: (pp[1][k] - mm[1][k]) / (2 * h) for k in xh}
    lhs = dot(ybs, jvp_s) + dot(ybh, jvp_h)
    rhs = dot(xbs, dxs) + dot(xbh, dxh)
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_adjoint_matches_oracle_directional_derivatives(L, base):
    """16 seeded directions: <J^T ybar, dx> (GPU adjoint) against <ybar, J_oracle dx> (oracle, central differences)."""
    S, ctx, cfg, xs, xh = base
    rng = np.random.default_rng(3000)

    def oracle_map(st, hi):
        hist = dict(hi)
        hist.update(s=1, z1=hi["z1"], z2=hi["z2"], z3=hi["z3"], zdot=hi["zdot"], r_om=hi["r_om"],
                    r_phi=hi["r_phi"], r_m1=hi["r_m"][:cfg.ny], r_m3=hi["r_m"][cfg.ny:])
        S.set_state(st["z"], st["om"], st["m2"], st["mm1"], st["mm3"], history=hist)
        S.advance_substage()
        h2 = S.history()
        out_h = dict(z1=h2["z1"], z2=h2["z2"], z3=h2["z3"], zdot=h2["zdot"], r_om=h2["r_om"], r_phi=h2["r_phi"],
                     r_m=np.concatenate([h2["r_m1"], h2["r_m3"]]))
        return S.state(), out_h

    ys, yh = oracle_map(xs, xh)
    ybs, ybh = _random_like(rng, cfg, ys, True), _random_like(rng, cfg, yh, False)
    xbs, xbh = _adjoint(L, ctx, cfg, xs, xh, ybs, ybh)
    h = 1e-6
    worst = 0.0
    for _ in range(16):
        dxs, dxh = _random_like(rng, cfg, xs, True), _random_like(rng, cfg, xh, False)
        pp = oracle_map({k: xs[k] + h * dxs[k] for k in xs}, {k: xh[k] + h * dxh[k] for k in xh})
        mm = oracle_map({k: xs[k] - h * dxs[k] for k in xs}, {k: xh[k] - h * dxh[k] for k in xh})
        lhs = dot(ybs, {k: (pp[0][k] - mm[0][k]) / (2 * h) for k in xs}) + \
            dot(ybh, {k: (pp[1][k] - mm[1][k]) / (2 * h) for k in xh})
        rhs = dot(xbs, dxs) + dot(xbh, dxh)
        worst = max(worst, abs(lhs - rhs) / max(abs(lhs), abs(rhs)))
    assert worst <= 1e-6, worst


# Cross blocks of the Jacobian with no identity part, so errors in the nonlinear pieces cannot hide
# behind the pass-through of z and of the history: (outputs weighted by ybar, inputs perturbed, step h).
# Blocks with h = 1e-3 are exactly affine in the perturbed inputs (z <- momentum: with z held, R_z is
# linear in m^d and the fixed point is affine in R_z; the RK update in RHS_prev and dz/dt_prev; the fixed
# point, with z held, in the BDF guess): there central differences have no truncation error, and the
# larger step keeps their rounding error small against the O(1) outputs they move by O(dt).
CROSS = [
    ("momentum <- z", {"om", "m2"}, set(), {"z"}, set(), 1e-6),                 # density, gravity, C_ij, u
    ("z <- momentum", {"z"}, set(), {"om", "m2", "mm1"}, set(), 1e-3),           # advection R_z, m^c
    ("zdot <- z", set(), {"zdot"}, {"z"}, set(), 1e-6),                          # fixed point, L(z), f'(z)
    ("rhs <- state", set(), {"r_om", "r_phi", "r_m"}, {"z", "om", "m2", "mm1", "mm3"}, set(), 1e-6),
    ("means <- momentum", {"mm1", "mm3"}, set(), {"om", "m2"}, set(), 1e-6),    # <C12>, <C23>
    ("state <- old rhs and zdot", {"z", "om", "m2", "mm1"}, set(), set(), {"r_om", "r_phi", "r_m", "zdot"}, 1e-3),
    ("zdot <- z history", set(), {"zdot"}, set(), {"z1", "z2", "z3"}, 1e-3),   # BDF guess through the iteration
]


def _seed(name):
    return zlib.crc32(name.encode())


@pytest.mark.parametrize("name,ys_keys,yh_keys,xs_keys,xh_keys,h", CROSS, ids=[c[0] for c in CROSS])
def test_adjoint_cross_blocks(L, base, name, ys_keys, yh_keys, xs_keys, xh_keys, h):
    S, ctx, cfg, xs, xh = base
    rng = np.random.default_rng(_seed(name))
    ys, yh = _gpu_map(L, ctx, cfg, xs, xh)
    ybs = {k: (v if k in ys_keys else 0 * v) for k, v in _random_like(rng, cfg, ys, True).items()}
    ybh = {k: (v if k in yh_keys else 0 * v) for k, v in _random_like(rng, cfg, yh, False).items()}
    dxs = {k: (v if k in xs_keys else 0 * v) for k, v in _random_like(rng, cfg, xs, True).items()}
    dxh = {k: (v if k in xh_keys else 0 * v) for k, v in _random_like(rng, cfg, xh, False).items()}
    xbs, xbh = _adjoint(L, ctx, cfg, xs, xh, ybs, ybh)
    pp = _gpu_map(L, ctx, cfg, {k: xs[k] + h * dxs[k] for k in xs}, {k: xh[k] + h * dxh[k] for k in xh})
    mm = _gpu_map(L, ctx, cfg, {k: xs[k] - h * dxs[k] for k in xs}, {k: xh[k] - h * dxh[k] for k in xh})
    lhs = dot(ybs, {k: (pp[0][k] - mm[0][k]) / (2 * h) for k in xs}) + \
        dot(ybh, {k: (pp[1][k] - mm[1][k]) / (2 * h) for k in xh})
    rhs = dot(xbs, dxs) + dot(xbh, dxh)
    assert abs(rhs) > 0
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs)), (name, lhs, rhs)


# ---- the start-up of lmvd_set_state without history: x -> (x, history), reading R6
def _startup_map(L, ctx, cfg, st):
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
    ctx.set_state(dev)
    hout = ctx.history_buffer()
    so = ctx.get_state(history=hout)
    ctx.synchronize()
    return {k: v.cpu().numpy() for k, v in so.items()}, unpack(cfg, hout.cpu().numpy(), "hist")


def _startup_adjoint(L, ctx, cfg, x_state, yb_state, yb_hist):
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in x_state.items()}
    ctx.set_state(dev)
    sbi = torch.zeros(L.lmvd_state_bytes(ctx.h), dtype=torch.uint8, device="cuda")
    sbo = torch.from_numpy(pack(cfg, yb_state, "state")).cuda()
    hbo = torch.from_numpy(pack(cfg, yb_hist, "hist")).cuda()
    L.lmvd_adjoint_startup(ctx.h, sbo, hbo, sbi)
    return unpack(cfg, sbi.cpu().numpy(), "state")


# (weighted outputs: state keys, history keys; perturbed state keys); the history-only blocks have no
# identity part (the state passes through the start-up unchanged)
STARTUP_BLOCKS = [
    ("all", {"z", "om", "m2", "mm1", "mm3"}, {"z1", "z2", "z3", "zdot"}, {"z", "om", "m2", "mm1", "mm3"}),
    ("history <- z", set(), {"z1", "z2", "z3", "zdot"}, {"z"}),
    ("history <- momentum", set(), {"z1", "z2", "z3", "zdot"}, {"om", "m2", "mm1", "mm3"}),
]


@pytest.mark.parametrize("name,ys_keys,yh_keys,xs_keys", STARTUP_BLOCKS, ids=[b[0] for b in STARTUP_BLOCKS])
def test_startup_adjoint_matches_gpu_central_differences(L, base, name, ys_keys, yh_keys, xs_keys):
    S, ctx, cfg, xs, _ = base
    rng = np.random.default_rng(_seed("startup " + name))
    ys, yh = _startup_map(L, ctx, cfg, xs)
    ybs = {k: (v if k in ys_keys else 0 * v) for k, v in _random_like(rng, cfg, ys, True).items()}
    ybh = {k: (v if k in yh_keys else 0 * v) for k, v in _random_like(rng, cfg, {**yh, **{
        q: np.ones_like(yh[q]) for q in ("r_om", "r_phi", "r_m")}}, False).items()}
    dxs = {k: (v if k in xs_keys else 0 * v) for k, v in _random_like(rng, cfg, xs, True).items()}
    xbs = _startup_adjoint(L, ctx, cfg, xs, ybs, ybh)
    h = 1e-6
    pp = _startup_map(L, ctx, cfg, {k: xs[k] + h * dxs[k] for k in xs})
    mm = _startup_map(L, ctx, cfg, {k: xs[k] - h * dxs[k] for k in xs})
    lhs = dot(ybs, {k: (pp[0][k] - mm[0][k]) / (2 * h) for k in xs}) + \
        dot(ybh, {k: (pp[1][k] - mm[1][k]) / (2 * h) for k in yh})
    rhs = dot(xbs, dxs)
    assert abs(rhs) > 0
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs)), (name, lhs, rhs)


def test_startup_adjoint_matches_oracle_directional_derivatives(L, base):
    """16 seeded directions: <J^T ybar, dx> (GPU) against the oracle's start-up by central differences."""
    S, ctx, cfg, xs, _ = base
    rng = np.random.default_rng(3100)

    def oracle_map(st):
        S.set_state(st["z"], st["om"], st["m2"], st["mm1"], st["mm3"])
        h2 = S.history()
        return S.state(), dict(z1=h2["z1"], z2=h2["z2"], z3=h2["z3"], zdot=h2["zdot"])

    ys, yh = oracle_map(xs)
    ybs = _random_like(rng, cfg, ys, True)
    ybh = _random_like(rng, cfg, yh, False)
    full_h = dict(ybh, r_om=np.zeros(ys["om"].shape, complex), r_phi=np.zeros(ys["m2"].shape, complex),
                  r_m=np.zeros(2 * cfg.ny))
    xbs = _startup_adjoint(L, ctx, cfg, xs, ybs, full_h)
    h = 1e-6
    worst = 0.0
    for _ in range(16):
        dxs = _random_like(rng, cfg, xs, True)
        pp = oracle_map({k: xs[k] + h * dxs[k] for k in xs})
        mm = oracle_map({k: xs[k] - h * dxs[k] for k in xs})
        lhs = dot(ybs, {k: (pp[0][k] - mm[0][k]) / (2 * h) for k in xs}) + \
            dot(ybh, {k: (pp[1][k] - mm[1][k]) / (2 * h) for k in yh})
        rhs = dot(xbs, dxs)
        worst = max(worst, abs(lhs - rhs) / max(abs(lhs), abs(rhs)))
    assert worst <= 1e-6, worst
