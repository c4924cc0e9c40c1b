#!/usr/bin/env python
"""Throughput of the variable-density pseudospectral substage on GB300.

Metric: Mpoints * RK-substages / s = nx * ny * nz * substages / time / 1e6 (unpadded grid; one
RK2 step = two substages). A bench "step" is one substage (Algorithm 2, steps 1-6) of the whole
field. Default workload: the 512 x 513 x 512 Rayleigh-Taylor-shaped state (density ratio 10,
interface modes |k| <= 32, rms 2e-3, Re 5000), plain FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

--impl cuda (default): the CUDA library through its C-ABI. `value` is timed with CUDA events on
the library's stream around K substages with the state resident in HBM (inputs are > 100 GB, far
larger than L2, so no flush is needed); `e2e` times the same substage through the public API with
pinned host buffers (state + history copied in and out every substage). Under torchrun each rank
runs an independent replica (the substage runs on one GPU, unsharded); `value` sums the work
of all ranks over the slowest rank's time.
--impl reference: the FP64 CPU oracle on the host cores, one bounded-sample substage per step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints*RK-substages/s"
UNIT = "Mpoints*substages/s"
# FP64 peak of GB300 from this pool's measurement: 0.596e12 DFMA/s at 1.99 GHz across 152 SMs is
# 2 DFMA/clk/SM; at the 2070 MHz maximum SM clock: 152 * 2 * 2 flop * 2.07e9 = 1.259 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64-equivalent peak of double-float arithmetic on the FP32 pipe: a radix-2 butterfly (10 classic
# flops: one complex multiply, two complex adds) costs 2 x 22 + 4 x 14 = 100 FP32 instructions in
# df64.h (TwoSum-renormalised adds, FMA TwoProd products), i.e. 10 instructions per classic flop;
# the FP32 pipe issues 152 SMs x 128 lanes x 2.07 GHz instructions per second.
DF64_EQ_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 10 / 1e12
# Measured DRAM bytes (read + write) of the dominant kernel class over its algorithmic bytes, from one ncu
# capture of a smaller case with the same transform length (512 x 33 x 512: 768-point x-transforms), keyed by
# (precision, kernel class, transform length). The class fft_x_inverse holds k_fft_x_inv (19042-19412 /
# 18826-19246 B per complex x-transform against 20480 algorithmic) and k_fft_x_inv_mul, whose epilogue also
# reads f' (30032-30297 / 29464-29716 B against 32768); over the 12 launches of one substage the measured
# bytes are these fractions of the
# algorithmic ones (profiles/fft_x_inverse_rt512y33_traffic.md). Full launches: the fraction times the
# launch's algorithmic bytes.
NCU_DRAM_FRACTION = {(0, "fft_x_inverse", 768): 0.9318, (1, "fft_x_inverse", 768): 0.9199}
CPU_SAMPLE_N = 128


def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GB300 (MEASURED_PEAKS.json), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("cuda", "reference"), default="cuda")
    ap.add_argument("--workload", default="rt512")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=0, help="0: FP64; 1: double-float transforms/products")
    ap.add_argument("--no-variant", action="store_true", help="skip timing the other precision")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward cost ratio")
    ap.add_argument("--adjoint-workload", default="rt128")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison of the transforms")
    ap.add_argument("--no-graphs", action="store_true", help="skip the eager / CUDA-graph comparison")
    ap.add_argument("--rates", action="store_true", help="print the issue rates of lmvd_rate_probe and exit")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(name):
    from paper_2206_09878_gb300.rt_inputs import WORKLOADS
    w = dict(WORKLOADS[name])
    return w, dict(workload="%s: %dx%dx%d FP64, density ratio %g, eta |k|<=%d rms %g, Re %g, dt %g"
                   % (name, w["nx"], w["ny"], w["nz"], w["ratio"], w["kmax"], w["eta_rms"], w["re"], w["dt"]),
                   grid=[w["nx"], w["ny"], w["nz"]], padded_grid=[3 * w["nx"] // 2, w["ny"], 3 * w["nz"] // 2],
                   spline_order=6, kf=4, l2="inputs larger than L2 (state > 100 GB); no flush")


# ------------------------------------------------------------------ oracle timing (host cores)
def oracle_rate(w, nsub, n=CPU_SAMPLE_N):
    """Time `nsub` oracle substages on an n x (n+1) x n grid of the same recipe; returns (Mpts*sub/s, cores, desc)."""
    from oracle import transforms
    from oracle.lmvd import Config, Substage
    from paper_2206_09878_gb300.rt_inputs import rt_state
    ws = dict(w)
    ws.update(nx=n, ny=n + 1, nz=n, kmax=max(1, w["kmax"] * n // w["nx"]))
    cfg = Config(nx=n, ny=n + 1, nz=n, re=ws["re"], rho_l=1.0 / ws["ratio"], dt=ws["dt"], n_startup=1)
    S = Substage(cfg)
    S.set_state(**rt_state(**ws))
    t0 = time.perf_counter()
    for _ in range(nsub):
        S.advance_substage()
    dt = time.perf_counter() - t0
    rate = n * (n + 1) * n * nsub / dt / 1e6
    desc = ("%d oracle substage(s) of the same recipe on a %dx%dx%d grid (start-up excluded), %.1f s"
            % (nsub, n, n + 1, n, dt))
    return rate, transforms.WORKERS, desc


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w, config = workload_config(args.workload)
    from oracle import transforms
    from oracle.lmvd import Config, Substage
    from paper_2206_09878_gb300.rt_inputs import rt_state
    n = CPU_SAMPLE_N
    wsm = dict(w)
    wsm.update(nx=n, ny=n + 1, nz=n, kmax=max(1, w["kmax"] * n // w["nx"]))
    cfg = Config(nx=n, ny=n + 1, nz=n, re=wsm["re"], rho_l=1.0 / wsm["ratio"], dt=wsm["dt"], n_startup=1)
    S = Substage(cfg)
    S.set_state(**rt_state(**wsm))
    for _ in range(args.warmup):
        S.advance_substage()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.advance_substage()
    el = time.perf_counter() - t0
    value = n * (n + 1) * n * args.steps / el / 1e6
    sample = ("each step is one oracle substage of the %s recipe on a %dx%dx%d grid (the full grid needs "
              "minutes per substage on the host)" % (args.workload, n, n + 1, n))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": transforms.WORKERS, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local].strip()
    return str(local)


# ------------------------------------------------------------------ multi-rank aggregation
def aggregate(ms_local, units_per_rank, world, device=None):
    """Slowest rank's time and the whole-job rate: value = units of all ranks / max time."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, units_per_rank * world / (ms_max / 1e3) / 1e6


# ------------------------------------------------------------------ CUDA arm
def time_variant(L, w, precision, args, stream, st_host, local, ws, e2e_steps=0):
    """Create a context, run warm-up + K timed substages (CUDA events on the library stream), read the
    per-class profile, optionally the end-to-end loop; return (result dict, final state on the host)."""
    import torch
    import torch.distributed as dist

    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"],
                                n_startup=4, precision=precision)
    ctx = L.Context(cfg, stream=stream)
    device_bytes = L.lmvd_device_bytes(ctx.h)
    ctx.set_state({k: v.cuda() for k, v in st_host.items()})
    torch.cuda.empty_cache()   # the staged input is no longer referenced
    for _ in range(args.warmup):
        ctx.advance_substage()
    ctx.synchronize()
    L.lmvd_profile_enable(ctx.h, True)
    launches0 = L.lmvd_kernel_launches(ctx.h)
    clocks = ClockSampler(gpu_index(local))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.advance_substage()
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = L.lmvd_kernel_launches(ctx.h) - launches0
    prof = {L.lmvd_kernel_class_name(c): L.lmvd_profile_read(ctx.h, c) for c in range(L.LMVD_KERNEL_CLASSES)}
    L.lmvd_profile_enable(ctx.h, False)
    final = {k: v.cpu() for k, v in ctx.get_state().items()}
    ctx.synchronize()
    torch.cuda.empty_cache()
    res = dict(ms=ms, clocks=ck, launches=launches, prof=prof, device_bytes=device_bytes)
    if e2e_steps > 0:
        host_in = {k: v.pin_memory() for k, v in st_host.items()}
        hist_dev = ctx.history_buffer()
        ctx.get_state(history=hist_dev)
        hist_in = hist_dev.cpu().pin_memory()
        host_out = ctx.empty_state("cpu", pin=True)
        hist_out = torch.empty_like(hist_in).pin_memory()
        ctx.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.set_state(host_in, history=hist_in)
            ctx.advance_substage()
            ctx.get_state(host_out, history=hist_out)
            ctx.synchronize()
        res["e2e_s"] = time.perf_counter() - t0
        res["e2e_bytes"] = sum(v.numel() * v.element_size() for v in host_in.values()) + hist_in.numel()
    ctx.close()
    return res, final


def traffic_per_launch(fp, kernel, grid, alg_bytes_per_launch):
    """DRAM bytes per launch from the ncu fraction of the algorithmic bytes (None where no capture matches)."""
    nx, _, nz = grid
    px = 3 * nx // 2
    frac = NCU_DRAM_FRACTION.get((fp, kernel, px))
    if frac is None or not alg_bytes_per_launch:
        return None
    return frac * alg_bytes_per_launch


def class_table(prof, steps):
    """Per kernel class and step: time, launches, algorithmic TFLOP/s and GB/s, and the GB/s as a fraction
    of the measured HBM copy bandwidth (prof: class -> (ms, launches, flops, bytes) over `steps` steps)."""
    peak = hbm_peak_gbs()[0]
    out = {}
    for k, (ms, n, fl, by) in prof.items():
        if n <= 0:
            continue
        gbs = by / (ms / 1e3) / 1e9 if ms > 0 else None
        out[k] = {"ms_per_step": ms / steps, "launches_per_step": n / steps,
                  "tflops": fl / (ms / 1e3) / 1e12 if ms > 0 else None,
                  "hbm_gbs": gbs, "hbm_frac": gbs / peak if gbs is not None else None}
    return out


def measured_rates(L, iters=4000):
    """Issue rates of this GPU from the library's probe (lmvd_rate_probe): FP64 FMA / add / multiply and
    FP32 FMA, operations per second (8 independent chains per thread, 8 CTAs of 256 per SM). The FP32 probe
    runs 50x the iterations, so that it too lasts ~10 ms and the launch costs < 0.1% of its time."""
    names = ("fp64_fma", "fp64_add", "fp64_mul", "fp32_fma")
    return {n: L.lmvd_rate_probe(op, iters * (50 if n == "fp32_fma" else 1)) for op, n in enumerate(names)}


def roofline_of(prof, ms_step_total, fp, grid, rates=None):
    """Dominant kernel class and its achieved algorithmic rate against the ALU peak of its arithmetic: the
    measured FMA rate (rates, from measured_rates) where given, else the figure derived from the SM count,
    2 DFMA (FP64) or 128 FFMA (FP32) per clock per SM and the 2.07 GHz maximum clock."""
    top = max(prof, key=lambda k: prof[k][0])
    tms, tn, tfl, tby = prof[top]
    achieved = tfl / (tms / 1e3) / 1e12 if tms > 0 else None
    if fp == 0 and rates:
        peak, note = 2.0 * rates["fp64_fma"] / 1e12, "FP64 peak measured: 2 flop x the FP64 FMA rate of lmvd_rate_probe"
    elif fp == 0:
        peak, note = FP64_PEAK_TFLOPS, "FP64 peak derived: 152 SMs x 2 DFMA/clk/SM (measured) x 2 flop x 2.07 GHz"
    elif rates:
        peak, note = rates["fp32_fma"] / 10.0 / 1e12, ("FP64-equivalent peak of double-float: the FP32 FMA rate of "
                                                       "lmvd_rate_probe / 10 FP32 instructions per classic flop")
    else:
        peak, note = DF64_EQ_PEAK_TFLOPS, ("FP64-equivalent peak of double-float on the FP32 pipe: 152 SMs x 128 "
                                            "lanes x 2.07 GHz / 10 FP32 instructions per classic flop")
    return {"kernel": top, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "traffic": traffic_per_launch(fp, top, grid, tby / tn if tn else None),
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic bytes of the "
                            "class on 512x33x512 (same 768-point transforms), times the average launch's "
                            "algorithmic bytes",
            "launches": int(tn), "algorithmic_bytes_per_launch": tby / tn if tn else None,
            "achieved_hbm_gbs": tby / (tms / 1e3) / 1e9 if tms > 0 else None, "peak_note": note,
            "share_of_step": tms / ms_step_total if ms_step_total > 0 else None}


def adjoint_ratio(L, name, stream, reps=3):
    """Cost of lmvd_adjoint_substage (which re-runs the forward substage with a tape) against one forward
    substage, FP64, on the given workload; CUDA events on the library stream, after one warm-up each."""
    import numpy as np
    import torch

    from paper_2206_09878_gb300.rt_inputs import rt_state
    w, _ = workload_config(name)
    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"],
                                n_startup=4)
    ctx = L.Context(cfg, stream=stream)
    ctx.set_state({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rt_state(**w).items()})
    ctx.advance_substage()
    hist = ctx.history_buffer()
    st = ctx.get_state(history=hist)
    sb = torch.zeros(L.lmvd_state_bytes(ctx.h), dtype=torch.uint8, device="cuda")
    hb_in = torch.zeros_like(hist)
    ybar_s = torch.ones(L.lmvd_state_bytes(ctx.h) // 8, dtype=torch.float64, device="cuda")
    ybar_h = torch.zeros_like(hist)
    ctx.synchronize()

    def timed(fn):
        fn()
        ctx.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def fwd():
        ctx.set_state(st, history=hist)
        ctx.advance_substage()

    def adj():
        ctx.set_state(st, history=hist)
        L.lmvd_adjoint_substage(ctx.h, ybar_s.view(torch.uint8), ybar_h, sb, hb_in)

    f_ms, a_ms = timed(fwd), timed(adj)
    ctx.close()
    return {"workload": "%s: %dx%dx%d FP64" % (name, w["nx"], w["ny"], w["nz"]), "forward_ms": f_ms,
            "adjoint_ms": a_ms, "ratio": a_ms / f_ms,
            "note": "adjoint_ms includes the forward substage it re-runs to record its tape",
            "gradient": gradient_ratio(L, name, stream)}


def cufft_comparison(L, w, stream, df_prof=None, steps=None, kf=4, reps=5):
    """Per-field time of the 3/2-rule synthesis and analysis at the bench grid: this library's FP64 passes
    (lmvd_inverse_transform / lmvd_forward_transform, 4 fields per call) and, as the comparison baseline,
    cuFFT through torch.fft in FP64 and FP32: irfft2 / rfft2 of the zero-padded field (padding outside the
    timed region), and the pruned pipeline (1D transforms along z over the retained columns only, then
    along x; the padding and truncation copies timed with it). The double-float per-field times come from the precision-1 run's kernel profile
    (8 + 4 (kf + 1) inverse and 12 + 2 kf forward fields per substage)."""
    import torch
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    px, pz, nxh = 3 * nx // 2, 3 * nz // 2, nx // 2 + 1
    cfg = L.lmvd_default_config(nx, ny, nz, n_startup=0)
    ctx = L.Context(cfg, stream=stream)
    nf = 4
    out = {}
    with torch.cuda.stream(stream):
        spec = torch.randn(nf, ny, nz, nxh, dtype=torch.complex128, device="cuda")
        phys = torch.empty(nf, ny, pz, px, dtype=torch.float64, device="cuda")

        def timed(fn, per):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps / per

        out["lmvd_fp64_inverse"] = timed(lambda: L.lmvd_inverse_transform(ctx.h, spec, phys, nf), nf)
        out["lmvd_fp64_forward"] = timed(lambda: L.lmvd_forward_transform(ctx.h, phys, spec, nf), nf)
        del spec, phys
        ctx.close()
        torch.cuda.empty_cache()
        for name, cdt, rdt in (("fp64", torch.complex128, torch.float64), ("fp32", torch.complex64, torch.float32)):
            padded = torch.randn(ny, pz, px // 2 + 1, dtype=cdt, device="cuda")
            real = torch.randn(ny, pz, px, dtype=rdt, device="cuda")
            # unnormalised both ways (no separate scaling kernel), the padding done outside the timed region:
            # cuFFT's most favourable form of the same synthesis / analysis
            out["cufft_%s_inverse" % name] = timed(lambda: torch.fft.irfft2(padded, s=(pz, px), norm="forward"), 1)
            out["cufft_%s_forward" % name] = timed(lambda: torch.fft.rfft2(real, norm="backward"), 1)
            del padded
            # pruned: batched 1D C2C transforms along z over the nx/2 retained kx columns only (the kz padding
            # written into a zero buffer, inside the timed region), then batched C2R along x with the kx
            # padding implicit (irfft's n = px); forward: R2C along x, the retained columns, C2C along z,
            # the retained kz rows gathered. This is the strongest cuFFT form of the same work.
            h = nz // 2
            spec_c = torch.randn(ny, nz, nxh, dtype=cdt, device="cuda")
            zbuf = torch.zeros(ny, pz, nx // 2, dtype=cdt, device="cuda")
            spec_o = torch.zeros(ny, nz, nxh, dtype=cdt, device="cuda")

            def pruned_inverse():
                zbuf[:, :h] = spec_c[:, :h, :nx // 2]
                zbuf[:, pz - h + 1:] = spec_c[:, h + 1:, :nx // 2]
                t = torch.fft.ifft(zbuf, dim=1, norm="forward")
                return torch.fft.irfft(t, n=px, dim=2, norm="forward")

            def pruned_forward():
                t = torch.fft.rfft(real, dim=2, norm="forward")[:, :, :nx // 2]
                u = torch.fft.fft(t, dim=1, norm="forward")
                spec_o[:, :h, :nx // 2] = u[:, :h]
                spec_o[:, h + 1:, :nx // 2] = u[:, pz - h + 1:]

            out["cufft_pruned_%s_inverse" % name] = timed(pruned_inverse, 1)
            out["cufft_pruned_%s_forward" % name] = timed(pruned_forward, 1)
            del real, spec_c, zbuf, spec_o
            torch.cuda.empty_cache()
    if df_prof and steps:
        n_inv, n_fwd = 8 + 4 * (kf + 1), 12 + 2 * kf
        out["lmvd_df_inverse"] = (df_prof["fft_z_inverse"][0] + df_prof["fft_x_inverse"][0]) / steps / n_inv
        out["lmvd_df_forward"] = (df_prof["fft_x_forward"][0] + df_prof["fft_z_forward"][0]) / steps / n_fwd
    return {"unit": "ms per field", "grid": [nx, ny, nz], "padded": [px, ny, pz], **out,
            "note": "cufft_*: whole padded field (irfft2 / rfft2); cufft_pruned_*: 1D C2C along z over the nx/2 "
                    "retained columns and C2R / R2C along x, padding and truncation copies included; this library "
                    "skips the zero padding and the truncated modes and pairs two real rows per complex transform"}


def graphs_comparison(L, stream, grids=((32, 33, 32), (64, 65, 64), (128, 129, 128)), substages=40):
    """ms per substage with eager launches and with CUDA-graph replay (lmvd_graphs_enable) on small,
    launch-bound grids (the 32 x 33 x 32 recipe, resized); 20 warm-up substages capture all 10 launch
    patterns first."""
    import numpy as np
    import torch
    from paper_2206_09878_gb300.rt_inputs import WORKLOADS, rt_state
    out = {}
    for nx, ny, nz in grids:
        w = dict(WORKLOADS["rt32"], nx=nx, ny=ny, nz=nz)
        row = {}
        for graphs in (False, True):
            cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"],
                                        dt=w["dt"], n_startup=4)
            ctx = L.Context(cfg, stream=stream)
            L.lmvd_graphs_enable(ctx.h, graphs)
            with torch.cuda.stream(stream):
                ctx.set_state({k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
                               for k, v in rt_state(**w).items()})
                for _ in range(20):
                    ctx.advance_substage()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(substages):
                    ctx.advance_substage()
                e1.record(stream)
                torch.cuda.synchronize()
            row["graph_ms" if graphs else "eager_ms"] = e0.elapsed_time(e1) / substages
            if graphs:
                row["graphs_held"] = L.lmvd_graph_count(ctx.h)
            ctx.close()
        out["%dx%dx%d" % (nx, ny, nz)] = row
    return out


def gradient_ratio(L, name, stream, rk_steps=20, every_steps=5):
    """The whole gradient of the adjoint configuration against its forward: start-up (n_startup = 20) and
    2 rk_steps substages from an initial state without history; the gradient runs that forward keeping a
    checkpoint every every_steps RK steps, then the adjoints (recomputing each segment) and the start-up
    adjoint. CUDA events on the library stream, on which the torch operations of the chain also run."""
    import numpy as np
    import torch

    from paper_2206_09878_gb300.autograd import Layout, Startup, Substages, state_from_dict
    from paper_2206_09878_gb300.rt_inputs import rt_state
    w, _ = workload_config(name)
    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"])
    ctx = L.Context(cfg, stream=stream)
    nsub, every = 2 * rk_steps, 2 * every_steps
    with torch.cuda.stream(stream):
        x0 = state_from_dict({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rt_state(**w).items()})
        lay = Layout(ctx)
        weight = torch.from_numpy(np.random.default_rng(0).normal(size=x0.numel())).cuda()

        def fwd():
            ctx.set_state({k: v for k, v in zip(("z", "om", "m2", "mm1", "mm3"), split(x0))})
            for _ in range(nsub):
                ctx.advance_substage()

        def split(x):
            u8 = x.view(torch.uint8)
            out = []
            for k in ("z", "om", "m2", "mm1", "mm3"):
                o, n = lay.off[k]
                out.append(u8[o:o + n])
            return out

        def grad():
            x = x0.clone().requires_grad_(True)
            s, h = Substages.apply(*Startup.apply(x, ctx), ctx, 0, nsub, every)
            (weight * s).sum().backward()

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        f_ms, g_ms = timed(fwd), timed(grad)
    ctx.close()
    return {"substages": nsub, "checkpoint_every_substages": every, "n_startup": cfg.n_startup,
            "forward_ms": f_ms, "gradient_ms": g_ms, "ratio": g_ms / f_ms,
            "note": "gradient_ms = forward with checkpoints + adjoints with segment recomputation + start-up adjoint"}


def rel_err(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def run_cuda(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2206_09878_gb300 import lmvd as L
    from paper_2206_09878_gb300.rt_inputs import rt_state

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w, config = workload_config(args.workload)
    config["parallelism"] = "replicas%d" % ws if ws > 1 else "single"
    config["precision"] = ("FP64 throughout" if args.precision == 0 else
                           "double-float transforms and products, FP64 spectral steps")
    npts = w["nx"] * w["ny"] * w["nz"]
    stream = torch.cuda.Stream()
    st = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in rt_state(**w).items()}

    rates = measured_rates(L)
    res, final = time_variant(L, w, args.precision, args, stream, st, local, ws, e2e_steps=args.e2e_steps)
    ms_max, value = aggregate(res["ms"], npts * args.steps, ws, device="cuda")
    prof = res["prof"]
    breakdown = class_table(prof, args.steps)
    e2e = None
    if args.e2e_steps > 0:
        e2e_value = aggregate(1e3 * res["e2e_s"], npts * args.e2e_steps, ws, device="cuda")[1]
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": res["e2e_bytes"],
               "d2h_bytes_per_step": res["e2e_bytes"], "steps": args.e2e_steps}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Rayleigh-Taylor-shaped state)", "config": config,
        "clocks": res["clocks"], "gpu_launches": int(res["launches"]),
        "device_bytes": res["device_bytes"],
        "roofline": roofline_of(prof, res["ms"], args.precision, (w["nx"], w["ny"], w["nz"]), rates), "e2e": e2e,
        "issue_rates": {**rates, "unit": "operations/s", "source": "lmvd_rate_probe before the timed region"},
        "kernels": breakdown,
        "hbm_peak": {"gbs": hbm_peak_gbs()[0], "source": hbm_peak_gbs()[1],
                     "note": "kernels[*].hbm_frac = algorithmic bytes / time / this copy bandwidth"},
    }
    if not args.no_variant:
        other = 1 - args.precision
        r2, f2 = time_variant(L, w, other, args, stream, st, local, ws)
        _, v2 = aggregate(r2["ms"], npts * args.steps, ws, device="cuda")
        errs = {k: rel_err(f2[k], final[k]) for k in ("z", "om", "m2")}
        out["variant"] = {
            "precision": ("FP64 throughout" if other == 0 else
                          "FP32-FFT: double-float (2 x FP32, error-free transformations) transforms and products, "
                          "FP64 solves / RHS / update"),
            "value": v2, "unit": UNIT, "ms_per_step": r2["ms"] / args.steps, "clocks": r2["clocks"],
            "device_bytes": r2["device_bytes"],
            "roofline": roofline_of(r2["prof"], r2["ms"], other, (w["nx"], w["ny"], w["nz"]), rates),
            "kernels": class_table(r2["prof"], args.steps),
            "state_rel_l2_vs_headline_after_%d_substages" % (args.warmup + args.steps): errs,
        }
    if rank == 0 and ws == 1 and not args.no_cufft:
        df_prof = prof if args.precision == 1 else (None if args.no_variant else r2["prof"])
        out["cufft_baseline"] = cufft_comparison(L, w, stream, df_prof, args.steps)
    if rank == 0 and ws == 1 and not args.no_graphs:
        out["graphs"] = graphs_comparison(L, stream)
    if rank == 0 and ws == 1 and not args.no_adjoint:
        out["adjoint"] = adjoint_ratio(L, args.adjoint_workload, stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, cores, desc = oracle_rate(w, 4)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def print_rates(iters):
    """The issue rates of this GPU (lmvd_rate_probe) with the SM clock sampled while they run."""
    import torch

    from paper_2206_09878_gb300 import lmvd as L
    torch.cuda.set_device(0)
    L.lmvd_rate_probe(0, 1000)   # module load and clock ramp
    sampler = ClockSampler(0)
    sampler.start()
    rates = {n: L.lmvd_rate_probe(op, iters) for op, n in enumerate(("fp64_fma", "fp64_add", "fp64_mul", "fp32_fma"))}
    clocks = sampler.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    per = {n: v / (sms * mhz * 1e6) for n, v in rates.items()}
    print(json.dumps({"unit": "operations/s", **rates, "per_clock_per_sm": per, "sms": sms, "iters": iters,
                      "clocks": clocks, "fp64_peak_tflops_at_sampled_clock": 2 * rates["fp64_fma"] / 1e12}))


def main():
    args = parse()
    if args.rates:
        print_rates(200000)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
