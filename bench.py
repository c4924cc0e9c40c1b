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
runs an independent replica (the substage is not sharded on one-GPU machines); `value` sums the work
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
# DRAM bytes per launch of the dominant kernel from one ncu capture (None until captured for this code)
NCU_TRAFFIC_PER_LAUNCH = None
CPU_SAMPLE_N = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("cuda", "reference"), default="cuda")
    ap.add_argument("--workload", default="rt512")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    npts = w["nx"] * w["ny"] * w["nz"]
    cfg = L.lmvd_default_config(w["nx"], w["ny"], w["nz"], re=w["re"], rho_light=1.0 / w["ratio"], dt=w["dt"],
                                n_startup=4)
    stream = torch.cuda.Stream()
    ctx = L.Context(cfg, stream=stream)
    st = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in rt_state(**w).items()}
    dev = {k: v.cuda() for k, v in st.items()}
    ctx.set_state(dev)
    for _ in range(args.warmup):
        ctx.advance_substage()
    ctx.synchronize()

    # ---- timed region: K substages, state resident in HBM
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
    ms_max, value = aggregate(ms, npts * args.steps, ws, device="cuda")

    # dominant kernel class: roofline (FFT passes are FP64-ALU bound on GB300)
    top = max(prof, key=lambda k: prof[k][0])
    tms, tn, tfl, tby = prof[top]
    achieved = tfl / (tms / 1e3) / 1e12 if tms > 0 else None
    roofline = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": NCU_TRAFFIC_PER_LAUNCH, "launches": int(tn),
                "algorithmic_bytes_per_launch": tby / tn if tn else None,
                "achieved_hbm_gbs": tby / (tms / 1e3) / 1e9 if tms > 0 else None,
                "peak_note": "FP64 peak derived: 152 SMs x 2 DFMA/clk/SM (measured) x 2 flop x 2.07 GHz",
                "share_of_step": tms / ms if ms > 0 else None}
    breakdown = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                     "tflops": (v[2] / (v[0] / 1e3) / 1e12) if v[0] > 0 else None,
                     "hbm_gbs": (v[3] / (v[0] / 1e3) / 1e9) if v[0] > 0 else None}
                 for k, v in prof.items() if v[1] > 0}

    # ---- end to end through the public API with pinned host buffers
    host_in = {k: v.pin_memory() for k, v in st.items()}
    hist_dev = ctx.history_buffer()
    ctx.get_state(history=hist_dev)
    hist_in = hist_dev.cpu().pin_memory()
    host_out = ctx.empty_state("cpu", pin=True)
    hist_out = torch.empty_like(hist_in).pin_memory()
    ctx.synchronize()
    state_bytes = sum(v.numel() * v.element_size() for v in host_in.values())
    hbytes = hist_in.numel()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.set_state(host_in, history=hist_in)
        ctx.advance_substage()
        ctx.get_state(host_out, history=hist_out)
        ctx.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = aggregate(1e3 * e2e_s, npts * args.e2e_steps, ws, device="cuda")[1] if args.e2e_steps > 0 else None
    ctx.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Rayleigh-Taylor-shaped state)", "config": config,
        "clocks": ck, "gpu_launches": int(launches), "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes + hbytes,
                "d2h_bytes_per_step": state_bytes + hbytes, "steps": args.e2e_steps},
        "kernels": breakdown,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, cores, desc = oracle_rate(w, 2)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
