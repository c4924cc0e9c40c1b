"""Long parity runs of the CUDA substage against the FP64 oracle on the large benchmark workloads.

Not collected by pytest (the oracle takes tens of minutes of host time here); run on a GPU machine:

  python tests/long_parity.py --workload rt256 --steps 20 --check 1 20 --out parity_rt256.json
  python tests/long_parity.py --workload rt512 --steps 1 --check 1 --out parity_rt512.json
  python tests/long_parity.py --workload rt256 --steps 20 --check 1 5 20 --sensitivity --no-gpu   # host only

For each RK step listed in --check (one step = two substages of Algorithm 2) it records the per-field
relative L2 error of the state (z, Omega2, m2^d and the whole m1, m3 momentum components) of the
FP64 GPU path and of the double-float precision path against the oracle, and of the double-float path
against the FP64 GPU path. The 256 x 257 x 256 workload is the 20-step density-ratio-25.7 case, the
512 x 513 x 512 one the precision variant's case. The seeded inputs are those of the tests.

--sensitivity runs the oracle a second time from the same state with z, Omega2 and m2^d multiplied by
1 + 2^-52 n (n standard normal, seed 7: about one rounding unit) and records that run's distance from
the first at the checked steps: the growth of one rounding error through the method, the scale against
which the GPU's distance from the oracle after many steps is read. --no-gpu skips the GPU runs.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="rt256")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--check", type=int, nargs="+", default=[1, 20])
    ap.add_argument("--out", default=None)
    ap.add_argument("--sensitivity", action="store_true")
    ap.add_argument("--no-gpu", action="store_true")
    args = ap.parse_args()

    import numpy as np

    from _pairs import compare_states, gpu_config, oracle_config, to_numpy, to_torch, workload
    from oracle.lmvd import Substage
    from paper_2206_09878_gb300.rt_inputs import rt_state

    w = workload(args.workload)
    cfg = oracle_config(w)
    st = rt_state(**w)
    checks = sorted(set(c for c in args.check if 1 <= c <= args.steps))
    # GPU first (both precisions), keeping the states at the checked steps on the host
    gpu = {0: {}, 1: {}}
    t0 = time.time()
    for precision in (() if args.no_gpu else (0, 1)):
        import torch

        from paper_2206_09878_gb300 import lmvd as L
        ctx = L.Context(gpu_config(L, cfg, precision))
        ctx.set_state(to_torch(st))
        for step in range(1, args.steps + 1):
            ctx.advance_substage()
            ctx.advance_substage()
            if step in checks:
                gpu[precision][step] = to_numpy(ctx.get_state())
        ctx.synchronize()
        assert L.lmvd_status(ctx.h) == 0
        ctx.close()
        torch.cuda.empty_cache()
    t_gpu = time.time() - t0
    # the oracle
    t0 = time.time()
    S = Substage(cfg)
    S.set_state(**st)
    if args.sensitivity:
        rng = np.random.default_rng(7)
        sp = dict(st)
        for k in ("z", "om", "m2"):
            sp[k] = st[k] * (1 + 2.0 ** -52 * rng.standard_normal(st[k].shape))
        S2 = Substage(cfg)
        S2.set_state(**sp)
    out = {"workload": args.workload, "grid": [cfg.nx, cfg.ny, cfg.nz], "density_ratio": w["ratio"],
           "re": cfg.re, "dt": cfg.dt, "steps": {}, "gpu_seconds": t_gpu}
    for step in range(1, args.steps + 1):
        S.step(1)
        if args.sensitivity:
            S2.step(1)
        if step in checks:
            ora = S.state()
            rec = {}
            if not args.no_gpu:
                rec = {"fp64_vs_oracle": compare_states(S, gpu[0][step], ora),
                       "df_vs_oracle": compare_states(S, gpu[1][step], ora),
                       "df_vs_fp64": compare_states(S, gpu[1][step], gpu[0][step])}
                rec["fp64_max"] = max(rec["fp64_vs_oracle"].values())
                rec["df_max"] = max(rec["df_vs_oracle"].values())
            if args.sensitivity:
                rec["perturbed_oracle_vs_oracle"] = compare_states(S, S2.state(), ora)
                rec["perturbed_max"] = max(rec["perturbed_oracle_vs_oracle"].values())
            out["steps"][str(step)] = rec
            print("step", step, json.dumps(rec), flush=True)
    out["oracle_seconds"] = time.time() - t0
    out["cores"] = os.cpu_count()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "steps"}))


if __name__ == "__main__":
    main()
