"""GPU: gradients through several substages with checkpointing (paper_2206_09878_gb300.autograd).

Loss: a weighted quadratic energy of the final momentum coefficients (Omega2, m2^d) and of z, after
6 substages of rt32. Checked against central differences on 4 seeded directions, and the gradient must
not depend on the checkpoint spacing (recomputation is deterministic).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available()
    from _pairs import make_pair, to_torch
    from paper_2206_09878_gb300 import lmvd as L
    from paper_2206_09878_gb300.autograd import Layout, get_state
    S, ctx, st, cfg = make_pair(L, "rt32", u_rms=1e-2)
    ctx.set_state(to_torch(st))
    lay = Layout(ctx)
    state, hb = get_state(ctx, lay, torch.device("cuda"))
    hist = hb[16:].view(torch.float64).clone()
    return ctx, lay, state, hist


def loss_of(lay, s):
    z, om, m2 = (s[slice(*_rng(lay, k))] for k in ("z", "om", "m2"))
    return 1e6 * (om ** 2).sum() + 1e6 * (m2 ** 2).sum() + 1e-3 * (z ** 2).sum()


def _rng(lay, k):
    """float64 index range of one field of the packed state."""
    o, n = lay.off[k]
    return o // 8, (o + n) // 8


def run(ctx, lay, state, hist, every, grad=True):
    from paper_2206_09878_gb300.autograd import Substages
    s = state.clone().requires_grad_(grad)
    h = hist.clone().requires_grad_(grad)
    out_s, out_h = Substages.apply(s, h, ctx, 0, 6, every)
    loss = loss_of(lay, out_s)
    if grad:
        loss.backward()
        return float(loss.detach()), s.grad.clone(), h.grad.clone()
    return float(loss)


def test_gradient_matches_central_differences(setup):
    ctx, lay, state, hist = setup
    loss, gs, gh = run(ctx, lay, state, hist, every=2)
    rng = np.random.default_rng(4)
    for _ in range(4):
        ds = torch.from_numpy(rng.normal(size=state.numel())).cuda() * state.abs().mean()
        dh = torch.from_numpy(rng.normal(size=hist.numel())).cuda() * hist.abs().mean()
        h = 1e-6
        lp = run(ctx, lay, state + h * ds, hist + h * dh, 6, grad=False)
        lm = run(ctx, lay, state - h * ds, hist - h * dh, 6, grad=False)
        fd = (lp - lm) / (2 * h)
        ad = float((gs * ds).sum() + (gh * dh).sum())
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), abs(ad)), (fd, ad)


def test_checkpoint_spacing_does_not_change_gradient(setup):
    ctx, lay, state, hist = setup
    _, g2, h2 = run(ctx, lay, state, hist, every=2)
    _, g6, h6 = run(ctx, lay, state, hist, every=6)
    assert torch.equal(g2, g6) and torch.equal(h2, h6)


def test_gradient_with_graph_replay_on_a_side_stream(setup):
    """The same gradient from a context on a side stream, where the forward substages (the checkpointed
    run and the segment recomputations) replay CUDA graphs and only the adjoint's recording runs eagerly:
    bit for bit the gradient of the legacy-stream context, which launches everything eagerly. It also
    checks that lmvd_set_state reads the counter of a history blob written on that stream a moment before
    in stream order (a read on the legacy stream saw a stale counter and ran the wrong RK stage)."""
    from _pairs import make_pair
    from paper_2206_09878_gb300 import lmvd as L
    from paper_2206_09878_gb300.autograd import Layout
    ctx, lay, state, hist = setup
    _, g_ref, h_ref = run(ctx, lay, state, hist, every=2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        _, ctx2, _, _ = make_pair(L, "rt32", u_rms=1e-2)   # created on the current (side) stream
        lay2 = Layout(ctx2)
        _, g2, h2 = run(ctx2, lay2, state, hist, every=2)
        held = L.lmvd_graph_count(ctx2.h)
        torch.cuda.synchronize()
        ctx2.close()
    assert held > 0
    assert torch.equal(g_ref, g2) and torch.equal(h_ref, h2)
