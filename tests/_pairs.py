"""Helpers shared by the GPU tests: build the oracle and the CUDA path on the same seeded input."""
import contextlib
import copy

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


# ---- intermediate fields of one substage ------------------------------------------------------

U64 = 2.0 ** -53          # unit roundoff of FP64
UNIT_ROUNDOFF = {0: U64, 1: 2.0 ** -48}   # FP64; double-float transforms and products (precision 1)
GUESS_WEIGHT = 8          # max over both stages of sum |a_i| of the guess coefficients (Eq. dzdt_guesses:
                          # (2, -2, 0, 0) at stage n, (0, 3, -4, 1) at stage ' with beta' = -4)
STATE_ULPS = 16           # relative error of a state field z, in units of U64 (state parity: <= 1e-15)
ITERATION_GROWTH = 2      # transient growth of an error through the k_f fixed-point applications: the
                          # iteration contracts only asymptotically (Sec. 3.1, Eq. y_k_delta: error L^k e0)
NOISE_MARGIN = 8          # bound / rounding-model spread
INTERMEDIATES = ("zdot", "Rz", "rho_t", "mc1", "mc2", "mc3", "R_om", "R_phi", "R_m")
DOWNSTREAM = ("rho_t", "mc1", "mc2", "mc3", "R_om", "R_phi", "R_m")
PLAIN_TOL = 1e-12


def oracle_intermediates(S):
    """The intermediate fields of the substage the oracle just took (copies)."""
    t = S.trace
    r_om, r_phi, r_m1, r_m3 = t["R"]
    return dict(zdot=t["zdot"].copy(), Rz=S.Rz.copy(), rho_t=t["rho_t"].copy(), mc1=t["mc"][0].copy(),
                mc2=t["mc"][1].copy(), mc3=t["mc"][2].copy(), R_om=r_om.copy(), R_phi=r_phi.copy(),
                R_m=np.concatenate([r_m1, r_m3]), z_prev=S.zh[0].copy())


def oracle_downstream(S, zdot):
    """The oracle's own steps after the fixed point, applied to a given dz/dt^{k_f} (the GPU's):
    rho_t (Sec. 4.3), m^c (Eq. COM_fourier .. mc_mean), pass 2 and the right-hand sides (Eq. DNS_system).
    Uses the pass-1 fields of the substage the oracle just took; changes nothing in S."""
    rt = S.rho_t(zdot)
    mc = S.mc_from_rhot(rt)
    r_om, r_phi, r_m1, r_m3 = S.rhs(S.physical_pass_2(mc))
    return dict(rho_t=rt, mc1=mc[0], mc2=mc[1], mc3=mc[2], R_om=r_om, R_phi=r_phi, R_m=np.concatenate([r_m1, r_m3]))


def oracle_rz(S, state):
    """The oracle's pass 1 (Sec. 2.1) on a given state, e.g. the GPU's at the start of the substage: its
    R_z (the right-hand side of the fixed point). Uses S's operators; changes nothing in S."""
    op = S.op
    T = copy.copy(S)
    T.trace = {}
    T.z = np.asarray(state["z"], dtype=np.complex128) * op.keep
    T.om = np.asarray(state["om"], dtype=np.complex128) * op.kmask
    T.m2 = np.asarray(state["m2"], dtype=np.complex128) * op.kmask
    T.mm1 = np.asarray(state["mm1"], dtype=np.float64)
    T.mm3 = np.asarray(state["mm3"], dtype=np.float64)
    T.physical_pass_1()
    return T.Rz


@contextlib.contextmanager
def rounding_model(S, u, seed):
    """Run the oracle as if every transform and every band evaluation rounded its result normwise:
    each output plane of a transform gets random noise of size u times its own rms, each band
    evaluation (B^(d) applied along y) noise of size u times |B^(d)| |input| (the rounding error of a
    sum of products). Test infrastructure around the oracle; nothing in it is changed."""
    import oracle.lmvd as ol
    rng = np.random.default_rng(seed)
    op = S.op
    phys0, spec0, ax0 = op.phys, op.spectral, ol._ax0

    def plane_noise(a):
        rms = np.sqrt(np.mean(np.abs(a) ** 2, axis=tuple(range(1, a.ndim)), keepdims=True))
        n = rng.standard_normal(a.shape)
        if np.iscomplexobj(a):
            n = (n + 1j * rng.standard_normal(a.shape)) / np.sqrt(2)
        return u * rms * n

    def phys(F):
        f = phys0(F)
        return f + plane_noise(f)

    def spectral(f):
        F = spec0(f)
        return (F + plane_noise(F)) * op.keep

    def ax0_noisy(A, F):
        out = ax0(A, F)
        mag = ax0(abs(A), np.abs(F))
        n = rng.standard_normal(out.shape)
        if np.iscomplexobj(out):
            n = (n + 1j * rng.standard_normal(out.shape)) / np.sqrt(2)
        return out + u * mag * n

    op.phys, op.spectral, ol._ax0 = phys, spectral, ax0_noisy
    try:
        yield
    finally:
        del op.phys, op.spectral
        ol._ax0 = ax0


def downstream_floor(S, zdot, draws=2):
    """Relative spread of each downstream field under the FP64 rounding model (max over draws)."""
    ref = oracle_downstream(S, zdot)
    floor = {k: 0.0 for k in DOWNSTREAM}
    for d in range(draws):
        with rounding_model(S, U64, 1234 + d):
            noisy = oracle_downstream(S, zdot)
        for k in DOWNSTREAM:
            floor[k] = max(floor[k], rel(noisy[k], ref[k]))
    return ref, floor


def gpu_intermediates(L, ctx):
    """The same fields read from the context through lmvd_get_field."""
    f = {"zdot": L.LMVD_FIELD_ZDOT, "Rz": L.LMVD_FIELD_RZ, "rho_t": L.LMVD_FIELD_RHO_T, "mc1": L.LMVD_FIELD_MC1,
         "mc2": L.LMVD_FIELD_MC2, "mc3": L.LMVD_FIELD_MC3, "R_om": L.LMVD_FIELD_R_OMEGA2,
         "R_phi": L.LMVD_FIELD_R_PHI2, "R_m": L.LMVD_FIELD_R_MEANS}
    return {k: ctx.field(v).cpu().numpy() for k, v in f.items()}


def guess_amplification(cfg, inter):
    """A = |z| / (dt |dz/dt|): how much the guess (a difference of z history divided by dt) magnifies
    a relative error of z, measured against dz/dt itself (Sec. 3.3.1: the 1/dt round-off floor)."""
    return np.linalg.norm(inter["z_prev"]) / (cfg.dt * np.linalg.norm(inter["zdot"]))


def zdot_tolerance(cfg, inter, precision=0):
    """Relative L2 bound for dz/dt^{k_f}.

    dt dz/dt^0 = sum_i a_i z^{s-i} with sum |a_i| <= GUESS_WEIGHT, each z^{s-i} carrying a relative error
    <= STATE_ULPS u, so |d(dz/dt^0)| <= 128 u |z| / dt; the k_f fixed-point applications carry it on as
    L^{k_f} times it, which may grow it transiently (ITERATION_GROWTH). Relative to dz/dt: 256 u A,
    A = |z| / (dt |dz/dt|); never below 1e-12 scaled by the arithmetic's unit roundoff (the transforms inside
    the iteration)."""
    plain = PLAIN_TOL * UNIT_ROUNDOFF[precision] / U64
    return max(plain, GUESS_WEIGHT * STATE_ULPS * ITERATION_GROWTH * U64 * guess_amplification(cfg, inter))


def intermediate_check(S, cfg, gpu, ora, precision=0, floor=None, state=None):
    """Errors and bounds of every intermediate of one substage.

    dz/dt is held to the oracle's own within zdot_tolerance. R_z comes from the state alone (pass 1); with
    `state` (the GPU's state at the start of the substage) it is held to the oracle's pass 1 applied to that
    state (oracle_rz), else to the oracle's own R_z, within 1e-12 scaled by the unit roundoff: past the
    first substage the two states differ by their own rounding, which a cancellation in R_z can amplify
    (the paper's symmetric set-up at 128 x 512 x 128). rho_t, m^c and the right-hand sides are
    linear maps of dz/dt that do not preserve relative errors, so they are held to the oracle's steps
    applied to the GPU's own dz/dt (oracle_downstream): each step checked on the same input. Their bound is
    NOISE_MARGIN times the spread of the rounding model (downstream_floor, FP64 unit roundoff, scaled to
    the precision's), never below the scaled 1e-12: the d^3/dy^3 evaluation in RHS_phi2 and the cancellation
    in the plane-mean right-hand sides put their floors above 1e-12 on some grids."""
    scale = UNIT_ROUNDOFF[precision] / U64
    down = oracle_downstream(S, gpu["zdot"])
    if floor is None:
        _, floor = downstream_floor(S, ora["zdot"])
    err, tol = {}, {}
    err["zdot"], tol["zdot"] = rel(gpu["zdot"], ora["zdot"]), zdot_tolerance(cfg, ora, precision)
    rz_ref = ora["Rz"] if state is None else oracle_rz(S, state)
    err["Rz"], tol["Rz"] = rel(gpu["Rz"], rz_ref), PLAIN_TOL * scale
    for k in DOWNSTREAM:
        err[k] = rel(gpu[k], down[k])
        tol[k] = max(PLAIN_TOL, NOISE_MARGIN * floor[k]) * scale
    return err, tol


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
