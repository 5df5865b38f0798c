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
    """Small volume, then the 145x174x145 volume, then the small one again: the
    third call runs in scratch that the large call filled with finite data, and
    the small volume's row padding differs from the large one's, so an element
    read before it is written would show as a difference.  Both runs use the
    same kernels as the context blur, so every output must equal it bit for bit."""
    from paper_2112_10258_gb300 import capi
    from workloads.volumes import blob_volume, brain_like_volume
    det = S.Sift3D()
    stream = torch.cuda.current_stream().cuda_stream
    small = (blob_volume(seed=9, shape=(37, 29, 23)), 1.2263)
    large = (brain_like_volume(seed=4), 2.4525)
    for vol, sigma in (small, large, small):
        d = torch.from_numpy(vol).cuda()
        nz, ny, nx = vol.shape
        ref = det.gaussian_blur(d, sigma)
        out = torch.full_like(d, float("nan"))
        rc = capi.sift3d_gaussian_blur_noalloc(d.data_ptr(), nx, ny, nz, sigma, 4.0, out.data_ptr(), stream)
        assert rc == capi.OK
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.array_equal(o, r), f"max difference {np.max(np.abs(o - r))} on {vol.shape}"
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
