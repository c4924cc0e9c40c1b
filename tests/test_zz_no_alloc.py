"""GPU: the allocation-free inverse transform against the context-based one.

lmvd_inverse_transform_noalloc serves callers that cannot allocate device memory (and so cannot create
a context); it keeps its working memory in a static per-device array. Here it is called twice in a row
with different inputs through the C-ABI and each output is compared with lmvd_inverse_transform on the
same input, at the tolerance of the other transform tests. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def _values(rng, nf, ny, nx, nz):
    f = rng.normal(size=(nf * ny, nz, nx))
    fh = np.fft.rfft2(f, axes=(1, 2), norm="forward")
    fh[:, nz // 2, :] = 0
    fh[:, :, nx // 2] = 0
    return torch.from_numpy(fh.reshape(nf, ny, nz, nx // 2 + 1)).cuda()


@pytest.mark.parametrize("nx,ny,nz,nf", [(32, 33, 32, 3), (128, 129, 128, 1), (24, 13, 16, 2)])
def test_two_calls_match_context_transform(L, nx, ny, nz, nf):
    rng = np.random.default_rng(7 + nx)
    ctx = L.Context(L.lmvd_default_config(nx, ny, nz))
    px, pz = 3 * nx // 2, 3 * nz // 2
    for call in range(2):                       # two calls in a row, different inputs
        spec = _values(rng, nf, ny, nx, nz)
        ref = torch.zeros((nf, ny, pz, px), dtype=torch.float64, device="cuda")
        out = torch.full_like(ref, float("nan"))
        L.lmvd_inverse_transform(ctx.h, spec, ref, nf)
        L.lmvd_inverse_transform_noalloc(nx, ny, nz, spec, out, nf)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= TOL, (call, err)
    ctx.close()


def test_rejects_grid_beyond_static_array(L):
    spec = torch.zeros(1, dtype=torch.complex128, device="cuda")
    phys = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmvdError) as e:
        L.lmvd_inverse_transform_noalloc(256, 257, 256, spec, phys, 1)
    assert e.value.code == -1
