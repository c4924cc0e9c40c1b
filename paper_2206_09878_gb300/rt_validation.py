"""Long-run validation on the paper's single-mode Rayleigh-Taylor set-up (Sec. 5).

Runs the CUDA substage from the paper's initial condition (tanh interface with h(x1, x3), potential
matching, W = g = 1) and records the bubble and spike heights
  h_b: where z = 1/2 on the vertical line through the highest point of the initial interface
       (x = z = 0; light fluid rising into heavy),
  h_s: where z = 1/2 on the line through the lowest point (x = z = 1/2 in 3D, x = 1/2 in 2D),
and the bubble velocity v_b = dh_b/dt. During the potential-growth phase v_b is near constant; the
paper compares it with Goncharov's potential-flow value (its Eq. potential_growth)
  v_b = sqrt(2 At / (1 + At) * g / (C k)),  k = 2 pi / W,  C = 1 in 3D, 3 in 2D.
A 2D case runs as a 3D grid with nz = 4 and an interface independent of z (modes with kz != 0 stay
exactly zero).

  python -m paper_2206_09878_gb300.rt_validation --dim 3 --at 0.5 --nx 64 --ny 257 --tend 5 --out run.json

All arithmetic of the method runs in the library; this module builds the initial state, samples z on
two vertical lines through spline evaluation (scipy) and reduces the samples.
"""
import argparse
import json
import math
import time

import numpy as np

from .rt_inputs import paper_dt


def goncharov(at, dim, g=1.0, wavelength=1.0):
    c = 1.0 if dim == 3 else 3.0
    k = 2 * math.pi / wavelength
    return math.sqrt(2 * at / (1 + at) * g / (c * k))


def initial_state(nx, ny, nz, y0, y1, dim, delta=0.0, eps=0.05):
    """z_hat of z = (1 + tanh((y - h) / (2 eps))) / 2 (spline coefficients = samples at uniform anchors,
    as in rt_inputs) and zero divergence-free momentum."""
    nxh = nx // 2 + 1
    x = np.arange(nx) / nx
    zc = np.arange(nz) / nz
    if dim == 3:
        h = 0.05 * (np.cos(2 * np.pi * x)[None, :] + np.cos(2 * np.pi * zc)[:, None]) + delta
    else:
        h = 0.1 * np.cos(2 * np.pi * x)[None, :] * np.ones((nz, 1)) + delta
    ya = y0 + (y1 - y0) * np.arange(ny) / (ny - 1)
    zf = 0.5 * (1 + np.tanh((ya[:, None, None] - h[None]) / (2 * eps)))
    zh = np.fft.rfft2(zf, axes=(1, 2), norm="forward")
    zh[:, nz // 2] = 0
    zh[:, :, nx // 2] = 0
    return dict(z=zh, om=np.zeros_like(zh), m2=np.zeros((ny + 1, nz, nxh), complex), mm1=np.zeros(ny),
                mm3=np.zeros(ny))


class LineProbe:
    """z on the bubble and spike lines from the spectral B-spline coefficients of z."""

    def __init__(self, nx, ny, nz, y0, y1, dim, p=6, samples=8001):
        from scipy.interpolate import BSpline
        self.BSpline = BSpline
        nint = ny - p + 1
        self.t = np.concatenate([np.full(p - 1, y0), y0 + (y1 - y0) * np.arange(nint + 1) / nint,
                                 np.full(p - 1, y1)])
        self.k = p - 1
        self.y = np.linspace(y0, y1, samples)
        nxh = nx // 2 + 1
        w = np.where(np.arange(nxh) == 0, 1.0, 2.0)[None, :] * np.ones((nz, 1))
        kz = np.fft.fftfreq(nz, 1.0 / nz)
        sign = (-1.0) ** np.arange(nxh)[None, :] * ((-1.0) ** kz[:, None] if dim == 3 else np.ones((nz, 1)))
        self.wb = w
        self.ws = w * sign

    def crossings(self, zhat, weights):
        c = (zhat.real * weights[None]).sum((1, 2))
        v = self.BSpline(self.t, c, self.k)(self.y) - 0.5
        idx = np.nonzero(np.sign(v[:-1]) != np.sign(v[1:]))[0]
        return [float(self.y[j] - v[j] * (self.y[j + 1] - self.y[j]) / (v[j + 1] - v[j])) for j in idx]

    def heights(self, zhat):
        """(h_b, h_s): the highest crossing on the bubble line and the lowest on the spike line."""
        b = self.crossings(zhat, self.wb)
        s = self.crossings(zhat, self.ws)
        return (max(b) if b else float("nan")), (min(s) if s else float("nan"))


def plateau(t, hb, window=1.0):
    """Bubble velocity of the potential-growth phase: v_b = dh_b/dt (central differences), then the
    window of the given duration after the initial acceleration with the smallest relative spread of v_b;
    returns (mean v_b in it, its spread max-min, window start, window end)."""
    t = np.asarray(t)
    hb = np.asarray(hb)
    ok = np.isfinite(hb)
    t, hb = t[ok], hb[ok]
    v = np.gradient(hb, t)
    best = None
    for i in range(len(t)):
        j = np.searchsorted(t, t[i] + window)
        if j >= len(t):
            break
        seg = v[i:j + 1]
        if seg.mean() <= 0:
            continue
        spread = (seg.max() - seg.min()) / seg.mean()
        # only after the velocity has reached 80 % of its running maximum (end of the initial acceleration)
        if v[i] < 0.8 * v[:j + 1].max():
            continue
        if best is None or spread < best[0]:
            best = (spread, float(seg.mean()), float(seg.max() - seg.min()), float(t[i]), float(t[j]))
    if best is None:
        return float("nan"), float("nan"), float("nan"), float("nan")
    return best[1:]


def run(dim=3, at=0.5, nx=64, ny=257, nz=None, y0=-2.0, y1=2.0, delta=0.0, re=None, tend=5.0, sample_every=50,
        precision=0, device=0, log=None):
    import torch

    from . import lmvd as L
    nz = (nx if dim == 3 else 4) if nz is None else nz
    re = (1024.0 if dim == 3 else 3000.0) if re is None else re
    dt = paper_dt(dim, at)
    cfg = L.lmvd_default_config(nx, ny, nz, lx=1.0, lz=1.0, y0=y0, y1=y1, re=re, sc=1.0, fr=1.0, rho_heavy=1.0,
                                rho_light=(1 - at) / (1 + at), dt=dt, bc_mode=1, precision=precision)
    torch.cuda.set_device(device)
    ctx = L.Context(cfg)
    st = initial_state(nx, ny, nz, y0, y1, dim, delta)
    ctx.set_state({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()})
    probe = LineProbe(nx, ny, nz, y0, y1, dim)
    nsteps = int(round(tend / dt))
    rec_t, rec_b, rec_s = [], [], []
    t0 = time.time()
    done = 0
    while True:
        zhat = ctx.get_state()["z"].cpu().numpy()
        hb, hs = probe.heights(zhat)
        rec_t.append(done * dt)
        rec_b.append(hb)
        rec_s.append(hs)
        if log and len(rec_t) % 20 == 1:
            log("t=%.3f h_b=%.4f h_s=%.4f (%.0f s)" % (done * dt, hb, hs, time.time() - t0))
        if done >= nsteps or not (y0 < hs and hb < y1):
            break
        n = min(sample_every, nsteps - done)
        ctx.step(n)
        done += n
    ctx.synchronize()
    wall = time.time() - t0
    status = L.lmvd_status(ctx.h)
    ctx.close()
    vb, spread, ta, tb = plateau(rec_t, rec_b)
    vg = goncharov(at, dim)
    return dict(dim=dim, at=at, grid=[nx, ny, nz], domain_y=[y0, y1], re=re, dt=dt, precision=precision,
                steps=done, wall_s=wall, status=status, t=rec_t, h_b=rec_b, h_s=rec_s,
                v_b_plateau=vb, v_b_spread=spread, plateau_window=[ta, tb], v_goncharov=vg, ratio=vb / vg)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3, choices=(2, 3))
    ap.add_argument("--at", type=float, nargs="+", default=[0.5])
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--ny", type=int, default=257)
    ap.add_argument("--y0", type=float, default=-2.0)
    ap.add_argument("--y1", type=float, default=2.0)
    ap.add_argument("--delta", type=float, default=0.0)
    ap.add_argument("--tend", type=float, default=5.0)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--sample-every", type=int, default=50)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = []
    for at in a.at:
        r = run(dim=a.dim, at=at, nx=a.nx, ny=a.ny, y0=a.y0, y1=a.y1, delta=a.delta, tend=a.tend,
                precision=a.precision, sample_every=a.sample_every, log=lambda s: print(s, flush=True))
        print(json.dumps({k: r[k] for k in ("dim", "at", "grid", "steps", "wall_s", "status", "v_b_plateau",
                                            "v_b_spread", "plateau_window", "v_goncharov", "ratio")}), flush=True)
        out.append(r)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
