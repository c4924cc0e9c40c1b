"""torch.autograd bridge: K substages of the CUDA path as one differentiable operation.

`Substages.apply(state, history, context, nsub, every)` advances a context by `nsub` substages from a
(state, history) pair given as flat float64 CUDA tensors (the packed state blob of lmvd_state_bytes and
the history blob of lmvd_history_bytes without its 16-byte counter header, viewed as float64), and
returns the final pair in the same form. Its backward pass calls lmvd_adjoint_substage once per
substage in reverse order. Memory is bounded by checkpointing: the forward keeps (state, history) every
`every` substages; the backward recomputes each segment from its checkpoint and runs the adjoints of
that segment from its last substage back to its first.

`Startup.apply(state, context)` is the start-up of lmvd_set_state without history as a differentiable
map state -> (state, history); its backward pass calls lmvd_adjoint_startup. Composed,
`Substages.apply(*Startup.apply(x, ctx), ctx, 0, nsub, every)` differentiates K substages from an
initial state that has no history.

All arithmetic runs in the library; this module only schedules calls and moves buffers. Gradients are
with respect to the real inner product of the stored entries (real and imaginary parts as separate
reals), i.e. the gradient of a real loss with respect to the float64 views.
"""
import numpy as np
import torch

from . import lmvd as L


class Layout:
    """Byte offsets of the packed state blob and sizes of the blobs of one context."""

    def __init__(self, ctx):
        cfg = ctx.cfg
        ny, nz, nxh = cfg.ny, cfg.nz, cfg.nx // 2 + 1
        s, sp, r = 16 * ny * nz * nxh, 16 * (ny + 1) * nz * nxh, 8 * ny
        self.off = dict(z=(0, s), om=(s, s), m2=(2 * s, sp), mm1=(2 * s + sp, r), mm3=(2 * s + sp + r, r))
        self.state_bytes = L.lmvd_state_bytes(ctx.h)
        self.hist_bytes = L.lmvd_history_bytes(ctx.h)
        assert self.state_bytes == 2 * s + sp + 2 * r


def history_blob(hist, s):
    """uint8 history blob: counter s, 8 bytes padding, then the float64 data."""
    blob = torch.empty(16 + hist.numel() * 8, dtype=torch.uint8, device=hist.device)
    blob[:16] = torch.from_numpy(np.array([s, 0], dtype=np.int64).view(np.uint8)).to(hist.device)
    blob[16:] = hist.contiguous().view(torch.uint8)
    return blob


def set_state(ctx, lay, state, hblob):
    """hblob None: the start-up runs (lmvd_set_state without history)."""
    u8 = state.contiguous().view(torch.uint8)
    v = {k: u8[o:o + n] for k, (o, n) in lay.off.items()}
    ctx.wait_inputs()
    L.lmvd_set_state(ctx.h, v["z"], v["om"], v["m2"], v["mm1"], v["mm3"], hblob)


def get_state(ctx, lay, dev):
    state = torch.empty(lay.state_bytes // 8, dtype=torch.float64, device=dev)
    hblob = torch.empty(lay.hist_bytes, dtype=torch.uint8, device=dev)
    u8 = state.view(torch.uint8)
    v = {k: u8[o:o + n] for k, (o, n) in lay.off.items()}
    ctx.wait_inputs()
    L.lmvd_get_state(ctx.h, v["z"], v["om"], v["m2"], v["mm1"], v["mm3"], hblob)
    ctx.publish()
    return state, hblob


def state_from_dict(st):
    """Pack a dict(z, om, m2, mm1, mm3) of CUDA tensors into the flat float64 state."""
    parts = [torch.view_as_real(st[k].contiguous()).reshape(-1) for k in ("z", "om", "m2")]
    parts += [st["mm1"].reshape(-1), st["mm3"].reshape(-1)]
    return torch.cat(parts)


class Substages(torch.autograd.Function):
    @staticmethod
    def forward(fctx, state, hist, ctx, s0, nsub, every):
        lay = Layout(ctx)
        dev = state.device
        hb = history_blob(hist, s0)
        ckpts = {0: (state.detach().clone(), hb.clone())}
        set_state(ctx, lay, state.detach(), hb)
        for j in range(1, nsub + 1):
            L.lmvd_advance_substage(ctx.h)
            if j % every == 0 and j < nsub:
                ckpts[j] = get_state(ctx, lay, dev)
        out_s, out_hb = get_state(ctx, lay, dev)
        ctx.synchronize()
        fctx.saved = (ctx, lay, ckpts, nsub, every)
        return out_s, out_hb[16:].view(torch.float64).clone()

    @staticmethod
    def backward(fctx, g_state, g_hist):
        ctx, lay, ckpts, nsub, every = fctx.saved
        dev = next(iter(ckpts.values()))[0].device
        ys = torch.zeros(lay.state_bytes // 8, dtype=torch.float64, device=dev) if g_state is None \
            else g_state.contiguous().clone()
        yh = history_blob(torch.zeros((lay.hist_bytes - 16) // 8, dtype=torch.float64, device=dev)
                          if g_hist is None else g_hist, 0)
        for start in sorted(ckpts, reverse=True):
            end = min(start + every, nsub)
            states = [ckpts[start]]
            set_state(ctx, lay, *ckpts[start])
            for _ in range(start + 1, end):
                L.lmvd_advance_substage(ctx.h)
                states.append(get_state(ctx, lay, dev))
            for xs, xh in reversed(states):
                set_state(ctx, lay, xs, xh)
                xbs = torch.empty_like(ys)
                xbh = torch.empty(lay.hist_bytes, dtype=torch.uint8, device=dev)
                ctx.wait_inputs()
                L.lmvd_adjoint_substage(ctx.h, ys.view(torch.uint8), yh, xbs.view(torch.uint8), xbh)
                ys, yh = xbs, xbh
        ctx.synchronize()
        return ys, yh[16:].view(torch.float64).clone(), None, None, None, None


class Startup(torch.autograd.Function):
    @staticmethod
    def forward(fctx, state, ctx):
        lay = Layout(ctx)
        x = state.detach().contiguous().clone()
        set_state(ctx, lay, x, None)
        out_s, out_hb = get_state(ctx, lay, state.device)
        ctx.synchronize()
        fctx.saved = (ctx, lay, x, out_hb)
        return out_s, out_hb[16:].view(torch.float64).clone()

    @staticmethod
    def backward(fctx, g_state, g_hist):
        ctx, lay, x, hb = fctx.saved
        dev = x.device
        ys = torch.zeros_like(x) if g_state is None else g_state.contiguous().clone()
        yh = history_blob(torch.zeros((lay.hist_bytes - 16) // 8, dtype=torch.float64, device=dev)
                          if g_hist is None else g_hist, 0)
        set_state(ctx, lay, x, hb)   # the state x; lmvd_adjoint_startup re-runs the start-up from it
        xb = torch.empty_like(x)
        ctx.wait_inputs()
        L.lmvd_adjoint_startup(ctx.h, ys.view(torch.uint8), yh, xb.view(torch.uint8))
        return xb, None
