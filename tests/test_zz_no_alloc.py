"""GPU: the allocation-free inverse transform.

lmvd_inverse_transform_noalloc serves callers that cannot allocate device memory (code running under
another framework's allocator, or after a start-up phase that forbids new allocations) and so cannot
create a context; it keeps its working memory in a static per-device array. Checks, through the C-ABI:
* two calls in a row with different inputs each match lmvd_inverse_transform on the same input and the
  oracle's 3/2-rule synthesis (oracle.transforms.to_phys), at the tolerance of the other transform tests;
* after the first call, a call allocates nothing: the device's free memory and the caching allocator's
  counters are the same before and after it;
* grids beyond the static array are rejected.

The file name puts it last in collection order: if it fails, a run that stops at the first failure has
already run every other test. It passes the same way alone in a fresh process (its first call on the
device does the set-up) and after the other tests (the array keeps the last call's contents, and every
call rewrites what it reads).
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
    return fh.reshape(nf, ny, nz, nx // 2 + 1)


@pytest.mark.parametrize("nx,ny,nz,nf", [(32, 33, 32, 3), (128, 129, 128, 1), (24, 13, 16, 2)])
def test_two_calls_match_context_transform_and_oracle(L, nx, ny, nz, nf):
    from oracle.transforms import to_phys
    rng = np.random.default_rng(7 + nx)
    ctx = L.Context(L.lmvd_default_config(nx, ny, nz))
    px, pz = 3 * nx // 2, 3 * nz // 2
    for call in range(2):                       # two calls in a row, different inputs
        spec_np = _values(rng, nf, ny, nx, nz)
        spec = torch.from_numpy(spec_np).cuda()
        ref = torch.zeros((nf, ny, pz, px), dtype=torch.float64, device="cuda")
        out = torch.full_like(ref, float("nan"))
        L.lmvd_inverse_transform(ctx.h, spec, ref, nf)
        L.lmvd_inverse_transform_noalloc(nx, ny, nz, spec, out, nf)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= TOL, (call, err)
        o = out.cpu().numpy()
        for f in range(nf):
            want = to_phys(spec_np[f], nx, nz)
            e = np.abs(o[f] - want).max() / np.abs(want).max()
            assert e <= TOL, (call, f, e)
    ctx.close()


def test_second_call_allocates_nothing(L):
    nx, ny, nz, nf = 64, 65, 64, 2
    rng = np.random.default_rng(11)
    spec = torch.from_numpy(_values(rng, nf, ny, nx, nz)).cuda()
    out = torch.empty((nf, ny, 3 * nz // 2, 3 * nx // 2), dtype=torch.float64, device="cuda")
    L.lmvd_inverse_transform_noalloc(nx, ny, nz, spec, out, nf)      # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    L.lmvd_inverse_transform_noalloc(nx, ny, nz, spec, out, nf)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


def test_rejects_grid_beyond_static_array(L):
    spec = torch.zeros(1, dtype=torch.complex128, device="cuda")
    phys = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LmvdError) as e:
        L.lmvd_inverse_transform_noalloc(256, 257, 256, spec, phys, 1)
    assert e.value.code == -1
