"""GPU: gradient of a kinetic-energy loss with respect to the initial interface amplitudes and the initial
momentum, through the start-up and K substages (lmvd_adjoint_startup + lmvd_adjoint_substage behind
paper_2206_09878_gb300.autograd.Startup and .Substages).

Parameters: the amplitudes a_k of the interface modes eta = sum a_k cos(kx x + kz z + theta_k) of the
seeded RT input (z follows through the generator's tanh profile, written in torch), and the initial
divergence-free momentum of the state (Omega2, m2^d and the plane means).
Loss: E = 1/2 int |m^d|^2 dV of the final state, the kinetic energy carried by the state's momentum
(the curl-free part m^c is not part of the state), evaluated exactly: Parseval in x and z, Gauss-Legendre
quadrature with p + 1 points per knot interval in y (exact for these piecewise polynomials).

Checks: central differences (h = 1e-6 relative) of the whole chain on the GPU, and, on the small case,
of the same chain with the oracle as the forward model. The adjoint configuration itself runs at
128 x 129 x 128: 20 RK steps (40 substages) at dt = 5e-4, checkpoints every 5 steps, 16 directions.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _quadrature(cfg):
    from oracle.bspline import Basis, collocation
    b = Basis(cfg.ny, cfg.p, cfg.y0, cfg.y1)
    br = np.unique(b.t)
    xg, wg = np.polynomial.legendre.leggauss(cfg.p + 1)
    yq = np.concatenate([0.5 * (r - l) * xg + 0.5 * (r + l) for l, r in zip(br[:-1], br[1:])])
    wq = np.concatenate([0.5 * (r - l) * wg for l, r in zip(br[:-1], br[1:])])
    return collocation(b.t, cfg.p, yq, 0), collocation(b.ts, cfg.p + 1, yq, 0), b.D, wq


class Energy:
    """E = 1/2 int |m^d|^2 dV of a state, with m1^d, m3^d from m2^d and Omega2 (Eq. md_recon)."""

    def __init__(self, cfg, device):
        Bq, Sq, D, wq = _quadrature(cfg)
        c128 = torch.complex128
        self.Bq = torch.as_tensor(Bq, dtype=c128, device=device)
        self.Sq = torch.as_tensor(Sq, dtype=c128, device=device)
        self.D = torch.as_tensor(D, dtype=c128, device=device)
        self.wq = torch.as_tensor(wq, dtype=torch.float64, device=device)
        nx, nz, nxh = cfg.nx, cfg.nz, cfg.nx // 2 + 1
        kx = np.arange(nxh) * 2 * np.pi / cfg.lx
        kz = np.fft.fftfreq(nz, 1.0 / nz) * 2 * np.pi / cfg.lz
        k1, k3 = np.meshgrid(kx, kz)
        keep = np.ones((nz, nxh))
        keep[nz // 2, :] = 0
        keep[:, nx // 2] = 0
        k2 = k1 ** 2 + k3 ** 2
        kmask = keep * (k2 > 0)
        safe = np.where(k2 > 0, k2, 1.0)
        self.a1 = torch.as_tensor(1j * k1 / safe * kmask, device=device)
        self.b1 = torch.as_tensor(-1j * k3 / safe * kmask, device=device)
        self.a3 = torch.as_tensor(1j * k3 / safe * kmask, device=device)
        self.b3 = torch.as_tensor(1j * k1 / safe * kmask, device=device)
        wk = np.where(np.arange(nxh)[None, :] == 0, 1.0, 2.0) * keep
        self.wk = torch.as_tensor(wk, device=device)
        self.vol = cfg.lx * cfg.lz
        self.cfg = cfg

    def fields(self, lay, s):
        cfg = self.cfg
        ny, nz, nxh = cfg.ny, cfg.nz, cfg.nx // 2 + 1

        def cplx(k, rows):
            o, n = lay.off[k]
            return torch.view_as_complex(s[o // 8:(o + n) // 8].reshape(rows, nz, nxh, 2))

        def real(k):
            o, n = lay.off[k]
            return s[o // 8:(o + n) // 8]
        return cplx("om", ny), cplx("m2", ny + 1), real("mm1"), real("mm3")

    def __call__(self, lay, s):
        om, m2, mm1, mm3 = self.fields(lay, s)
        dm2 = torch.einsum("ij,jab->iab", self.D, m2)
        m1 = self.a1 * dm2 + self.b1 * om
        m3 = self.a3 * dm2 + self.b3 * om
        mean = torch.zeros_like(m1)
        mean[:, 0, 0] = 1.0
        m1 = m1 + mean * mm1.to(torch.complex128)[:, None, None]
        m3 = m3 + mean * mm3.to(torch.complex128)[:, None, None]
        e = 0.0
        for B, f in ((self.Bq, m1), (self.Sq, m2), (self.Bq, m3)):
            v = torch.einsum("qj,jab->qab", B, f)
            e = e + (self.wq[:, None, None] * self.wk * (v.real ** 2 + v.imag ** 2)).sum()
        return 0.5 * self.vol * e


class Chain:
    """amplitudes, momentum -> initial state -> start-up -> nsub substages -> E, on the GPU."""

    def __init__(self, name, nsub, every, **over):
        from _pairs import make_pair
        from paper_2206_09878_gb300 import lmvd as L
        from paper_2206_09878_gb300.autograd import Layout
        from paper_2206_09878_gb300.rt_inputs import eta_modes
        self.S, self.ctx, st, self.cfg = make_pair(L, name, **over)
        from _pairs import workload
        self.w = workload(name, **{k: v for k, v in over.items() if k in workload(name)})
        self.lay = Layout(self.ctx)
        self.modes, self.theta, a = eta_modes(**self.w)
        dev = torch.device("cuda")
        self.amps0 = torch.full((len(self.modes),), a * self.w["eta_rms"], dtype=torch.float64, device=dev)
        parts = [torch.view_as_real(torch.from_numpy(st[k])).reshape(-1) for k in ("om", "m2")]
        parts += [torch.from_numpy(st["mm1"]), torch.from_numpy(st["mm3"])]
        self.vel0 = torch.cat(parts).to(dev)
        self.E = Energy(self.cfg, dev)
        self.nsub, self.every = nsub, every

    def state(self, amps, vel):
        from paper_2206_09878_gb300.rt_inputs import z_from_eta_torch
        z = z_from_eta_torch(amps, self.modes, self.theta, **self.w)
        return torch.cat([torch.view_as_real(z).reshape(-1), vel])

    def loss(self, amps, vel):
        from paper_2206_09878_gb300.autograd import Startup, Substages
        x = self.state(amps, vel)
        s0, h0 = Startup.apply(x, self.ctx)
        s, _ = Substages.apply(s0, h0, self.ctx, 0, self.nsub, self.every)
        return self.E(self.lay, s)

    def gradient(self):
        amps = self.amps0.clone().requires_grad_(True)
        vel = self.vel0.clone().requires_grad_(True)
        loss = self.loss(amps, vel)
        loss.backward()
        return float(loss.detach()), amps.grad.clone(), vel.grad.clone()

    def directions(self, rng):
        """Random directions over every stored entry: slots the method never reads (Nyquist, k = 0 of
        Omega2 and m2^d) are ignored by the forward and get zero gradient, so they cancel consistently."""
        da = torch.from_numpy(rng.normal(size=self.amps0.numel())).cuda() * self.amps0.abs().mean()
        dv = torch.from_numpy(rng.normal(size=self.vel0.numel())).cuda() * self.vel0.abs().mean()
        return da, dv


def _check_fd(chain, ndir, seed, forward=None, tol=1e-5):
    loss, ga, gv = chain.gradient()
    assert loss > 0
    rng = np.random.default_rng(seed)
    h = 1e-6
    worst = 0.0
    for _ in range(ndir):
        da, dv = chain.directions(rng)
        f = forward or (lambda a, v: float(chain.loss(a, v)))
        lp = f(chain.amps0 + h * da, chain.vel0 + h * dv)
        lm = f(chain.amps0 - h * da, chain.vel0 - h * dv)
        fd = (lp - lm) / (2 * h)
        ad = float((ga * da).sum() + (gv * dv).sum())
        worst = max(worst, abs(fd - ad) / max(abs(fd), abs(ad)))
    print("worst relative difference over %d directions: %.2e" % (ndir, worst))
    assert worst <= tol, worst
    return ga, gv


@pytest.fixture(scope="module")
def small():
    assert torch.cuda.is_available()
    return Chain("rt32", nsub=8, every=4, u_rms=1e-2)


def test_initial_condition_gradient_small_gpu(small):
    _check_fd(small, 8, 11)


def test_initial_condition_gradient_small_oracle(small):
    """The same chain with the FP64 oracle as the forward model (central differences on 4 directions)."""
    chain = small
    S, cfg, lay = chain.S, chain.cfg, chain.lay
    ny, nz, nxh = cfg.ny, cfg.nz, cfg.nx // 2 + 1

    def oracle_loss(a, v):
        x = chain.state(a, v).cpu()
        sl = {k: x[o // 8:(o + n) // 8].numpy() for k, (o, n) in lay.off.items()}
        cz = lambda k, r: sl[k].view(np.complex128).reshape(r, nz, nxh)
        S.set_state(cz("z", ny), cz("om", ny), cz("m2", ny + 1), sl["mm1"], sl["mm3"])
        for _ in range(chain.nsub):
            S.advance_substage()
        st = S.state()
        flat = np.concatenate([np.ascontiguousarray(st[k]).view(np.float64).ravel() for k in ("z", "om", "m2")]
                              + [st["mm1"], st["mm3"]])
        return float(chain.E(lay, torch.from_numpy(flat).cuda()))
    _check_fd(chain, 4, 12, forward=oracle_loss)


def test_adjoint_configuration_128():
    """128 x 129 x 128, 20 RK steps at dt = 5e-4, checkpoints every 5 steps, 16 directions."""
    chain = Chain("rt128", nsub=40, every=10)
    _check_fd(chain, 16, 13)
