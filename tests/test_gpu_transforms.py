"""GPU: the public 3/2-rule transforms (lmvd_inverse_transform / lmvd_forward_transform) against the
oracle's numpy transforms (Eq. disc_f, Sec. 4.4), on several grid shapes with ragged CTA batches."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def _random_values(rng, nf, ny, nx, nz):
    """Random real band-limited fields sampled on the unpadded grid -> retained spectral values."""
    f = rng.normal(size=(nf * ny, nz, nx))
    fh = np.fft.rfft2(f, axes=(1, 2), norm="forward")
    fh[:, nz // 2, :] = 0
    fh[:, :, nx // 2] = 0
    return fh.reshape(nf, ny, nz, nx // 2 + 1)


# (12, 13, 12): 18-point transforms in both directions, whose plans have no radix-4 stage (radices 2, 3, 3), so
# their first stage reads the zero padding band instead of pruning it
@pytest.mark.parametrize("nx,ny,nz,nf", [(32, 33, 32, 3), (24, 13, 16, 1), (64, 17, 8, 11), (128, 10, 96, 2),
                                         (12, 13, 12, 2)])
def test_inverse_and_forward_match_oracle(L, nx, ny, nz, nf):
    from oracle.transforms import to_phys, to_spec
    rng = np.random.default_rng(nx + ny + nz + nf)
    ctx = L.Context(L.lmvd_default_config(nx, ny, nz))
    spec = _random_values(rng, nf, ny, nx, nz)
    px, pz = 3 * nx // 2, 3 * nz // 2
    d_spec = torch.from_numpy(spec).cuda()
    d_phys = torch.zeros((nf, ny, pz, px), dtype=torch.float64, device="cuda")
    L.lmvd_inverse_transform(ctx.h, d_spec, d_phys, nf)
    back = torch.zeros_like(d_spec)
    L.lmvd_forward_transform(ctx.h, d_phys, back, nf)
    ctx.synchronize()
    phys = d_phys.cpu().numpy()
    for f in range(nf):
        ref = to_phys(spec[f], nx, nz)
        assert np.abs(phys[f] - ref).max() <= 1e-13 * np.abs(ref).max()
        refs = to_spec(ref, nx, nz)
        got = back[f].cpu().numpy()
        assert np.abs(got - refs).max() <= 1e-13 * np.abs(refs).max()
        assert np.abs(got - spec[f]).max() <= 1e-13 * np.abs(spec[f]).max()   # round trip
    ctx.close()
