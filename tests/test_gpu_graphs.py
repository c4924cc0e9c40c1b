"""GPU: substages replayed from CUDA graphs (lmvd_graphs_enable, on by default on a non-default stream).

A context captures each launch pattern of a substage once and replays it afterwards. The pattern is
the stage (n or ', Algorithm 2), the diagnostics flag and which buffer holds which state and history
field: z's history cycles through five buffers and the other fields through two, so 12 substages
visit all 10 patterns and replay two of them. Checked:
* the state after 12 substages equals bit for bit that of a context launching the same kernels eagerly
  (same kernels, arguments and order; no atomics touch the state), in both precisions, with the same
  kernel count;
* the replayed path matches the oracle at 1e-12 like the eager one;
* toggling diagnostics starts new patterns, and the record still matches the oracle's fixed-point
  changes; while profiling, launches are eager (per-launch CUDA events) and no graph is added.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NSUB = 12


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def _setup(L, precision, graphs, name="rt32"):
    """A context on the current (side) stream with graphs on or off, plus the oracle and the input."""
    from _pairs import gpu_config, oracle_config, workload
    from oracle.lmvd import Substage
    from paper_2206_09878_gb300.rt_inputs import rt_state
    w = workload(name)
    cfg = oracle_config(w)
    ctx = L.Context(gpu_config(L, cfg, precision))
    L.lmvd_graphs_enable(ctx.h, graphs)
    return Substage(cfg), ctx, rt_state(**w)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_eager_bitwise(L, precision):
    from _pairs import to_torch
    s = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(s):
        for graphs in (False, True):
            _, ctx, st = _setup(L, precision, graphs)
            ctx.set_state(to_torch(st))
            n0 = L.lmvd_kernel_launches(ctx.h)
            for _ in range(NSUB):
                ctx.advance_substage()
            n1 = L.lmvd_kernel_launches(ctx.h)
            state = {k: v.cpu() for k, v in ctx.get_state().items()}
            ctx.synchronize()
            out[graphs] = (state, n1 - n0, L.lmvd_graph_count(ctx.h))
            ctx.close()
    (eager, n_eager, g_eager), (graph, n_graph, g_graph) = out[False], out[True]
    assert g_eager == 0 and g_graph == 10, (g_eager, g_graph)
    assert n_eager == n_graph, (n_eager, n_graph)
    for k in eager:
        assert torch.equal(eager[k], graph[k]), k


def test_graph_replay_matches_oracle(L):
    from _pairs import compare_states, to_numpy, to_torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        S, ctx, st = _setup(L, 0, True)
        S.set_state(**st)
        ctx.set_state(to_torch(st))
        worst = 0.0
        for _ in range(NSUB):
            S.advance_substage()
            ctx.advance_substage()
            gpu = to_numpy(ctx.get_state())
            ctx.synchronize()
            worst = max(worst, max(compare_states(S, gpu, S.state()).values()))
        assert L.lmvd_graph_count(ctx.h) == 10
        ctx.close()
    assert worst <= 1e-12, worst


def test_diagnostics_and_profiling_with_graphs(L):
    from _pairs import to_torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        S, ctx, st = _setup(L, 0, True)
        S.set_state(**st)
        ctx.set_state(to_torch(st))
        S.advance_substage()
        ctx.advance_substage()
        assert L.lmvd_graph_count(ctx.h) == 1
        L.lmvd_diagnostics_enable(ctx.h, True)   # a new pattern: captured with the diagnostics launches
        S.advance_substage()
        ctx.advance_substage()
        assert L.lmvd_graph_count(ctx.h) == 2
        d = L.lmvd_diagnostics(ctx.h)
        assert d["substage"] == 1
        for g, o in zip(d["fp_changes"], S.fp_residuals):
            assert abs(g - o) <= 1e-3 * o + 1e-11, (g, o)
        L.lmvd_profile_enable(ctx.h, True)
        ctx.advance_substage()
        prof = [L.lmvd_profile_read(ctx.h, c) for c in range(L.LMVD_KERNEL_CLASSES)]
        L.lmvd_profile_enable(ctx.h, False)
        assert L.lmvd_graph_count(ctx.h) == 2          # profiled substages run eagerly
        assert sum(p[0] for p in prof) > 0 and sum(p[1] for p in prof) > 0
        assert L._lib.lmvd_synchronize(ctx.h) == 0
        ctx.close()


def test_substage_inside_a_callers_graph_capture(L):
    """A caller capturing the context's stream (torch.cuda.graph) gets the substage's launches in its own
    graph: the library does not start a capture of its own; one replay equals one eager substage."""
    from _pairs import to_torch
    s = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(s):
        for mode in ("eager", "caller_graph"):
            _, ctx, st = _setup(L, 0, mode != "eager")
            ctx.set_state(to_torch(st))
            ctx.advance_substage()
            if mode == "eager":
                ctx.advance_substage()
            else:
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    ctx.advance_substage()
                assert L.lmvd_graph_count(ctx.h) == 1        # only the substage before the capture
                g.replay()
            out[mode] = {k: v.cpu() for k, v in ctx.get_state().items()}
            ctx.synchronize()
            ctx.close()
    for k in out["eager"]:
        assert torch.equal(out["eager"][k], out["caller_graph"][k]), k
