"""Helpers shared by the GPU tests: build the oracle and the CUDA path on the same seeded input."""
import numpy as np
import torch

from oracle.lmvd import Config, Substage
from paper_2206_09878_gb300.rt_inputs import PAPER_RT, WORKLOADS, paper_rt_config, rt_paper_state, rt_state


def workload(name, **over):
    w = dict(WORKLOADS[name])
    w.update(over)
    return w


def oracle_config(w, **over):
    c = dict(nx=w["nx"], ny=w["ny"], nz=w["nz"], p=w.get("p", 6), re=w["re"], rho_h=1.0,
             rho_l=1.0 / w["ratio"], dt=w["dt"], kf=w.get("kf", 4), n_startup=w.get("n_startup", 20))
    c.update(over)
    return Config(**c)


def gpu_config(L, cfg, precision=0, memory_layout=0):
    return L.lmvd_default_config(cfg.nx, cfg.ny, cfg.nz, spline_order=cfg.p, lx=cfg.lx, lz=cfg.lz, y0=cfg.y0,
                                 y1=cfg.y1, re=cfg.re, sc=cfg.sc, fr=cfg.fr, rho_heavy=cfg.rho_h,
                                 rho_light=cfg.rho_l, dt=cfg.dt, kf=cfg.kf, beta_n=cfg.beta_n,
                                 beta_p=cfg.beta_p, n_startup=cfg.n_startup, precision=precision,
                                 bc_mode=1 if cfg.bc == "potential" else 0, memory_layout=memory_layout)


def to_torch(st, device="cuda"):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in st.items()}


def to_numpy(st):
    return {k: v.detach().cpu().numpy() for k, v in st.items()}


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def momentum_components(S, st):
    """m1^d, m3^d (B coefficients incl. the plane means) of a state, via the oracle's Eq. md_recon."""
    return S.md_components(st["m2"], st["om"], st["mm1"], st["mm3"])


def compare_states(S, gpu, ora):
    """Per-field relative L2 errors of the state: z, Omega2, m2^d and the whole m1, m3 components."""
    e = {k: rel(gpu[k], ora[k]) for k in ("z", "om", "m2")}
    g1, g3 = momentum_components(S, gpu)
    o1, o3 = momentum_components(S, ora)
    e["m1"] = rel(g1, o1)
    e["m3"] = rel(g3, o3)
    return e


def make_pair(L, name, precision=0, memory_layout=0, **over):
    w = workload(name, **{k: v for k, v in over.items() if k in WORKLOADS[name]})
    cfg = oracle_config(w, **{k: v for k, v in over.items() if k not in WORKLOADS[name]})
    S = Substage(cfg)
    st = rt_state(**w)
    ctx = L.Context(gpu_config(L, cfg, precision, memory_layout))
    return S, ctx, st, cfg


def make_paper_pair(L, name, precision=0, **over):
    """The paper's own RT set-up (potential matching, tanh interface with h(x1, x3), zero m^d)."""
    w = dict(PAPER_RT[name])
    w.update({k: v for k, v in over.items() if k in w})
    c = paper_rt_config(**w)
    c.update({k: v for k, v in over.items() if k not in w})
    cfg = Config(**c)
    S = Substage(cfg)
    st = rt_paper_state(**w)
    ctx = L.Context(gpu_config(L, cfg, precision))
    return S, ctx, st, cfg
