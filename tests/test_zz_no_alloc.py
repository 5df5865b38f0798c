"""sift3d_gaussian_blur_noalloc: the blur for callers that cannot allocate device
memory (it runs on a library-owned device scratch array instead).  Its output
must equal the context-based sift3d_gaussian_blur on the same input, on two
calls in a row (the second reuses the scratch the first left behind).  This file
is collected last so a failure here cannot hide the other tests' results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def test_noalloc_blur_matches_context_blur_twice(S):
    from paper_2112_10258_gb300 import capi
    from workloads.volumes import blob_volume, brain_like_volume
    det = S.Sift3D()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(brain_like_volume(seed=4), 2.4525), (blob_volume(seed=9, shape=(37, 29, 23)), 1.2263)]
    for vol, sigma in cases:
        d = torch.from_numpy(vol).cuda()
        nz, ny, nx = vol.shape
        ref = det.gaussian_blur(d, sigma)
        out = torch.full_like(d, float("nan"))
        rc = capi.sift3d_gaussian_blur_noalloc(d.data_ptr(), nx, ny, nz, sigma, 4.0, out.data_ptr(), stream)
        assert rc == capi.OK
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) <= 1e-5 * np.max(np.abs(r))
    det.close()


def test_noalloc_rejects_volumes_beyond_the_scratch(S):
    from paper_2112_10258_gb300 import capi
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.zeros(8, dtype=torch.float32, device="cuda")
    # roundup(nx, 8) * ny * nz > 2^22 elements; checked before any device work
    assert capi.sift3d_gaussian_blur_noalloc(d.data_ptr(), 256, 256, 65, 1.5, 4.0, d.data_ptr(),
                                             stream) == capi.ECAPACITY
    assert capi.sift3d_gaussian_blur_noalloc(d.data_ptr(), 4, 4, 4, -1.0, 4.0, d.data_ptr(),
                                             stream) == capi.EINVAL
