"""Every entry point that writes into caller buffers stays inside the extent it
was given: each output buffer is followed by a guard region of canary bytes
that must come back unchanged (odd, ragged shapes; a capacity smaller than the
keypoint count).  The device writes are checked without a sanitizer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.volumes import blob_volume  # noqa: E402

GUARD = 4096   # bytes of canaries after every output
CANARY = 0xA5


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _guarded(nbytes):
    """A device byte buffer of nbytes followed by the guard region."""
    t = torch.full((nbytes + GUARD,), CANARY, dtype=torch.uint8, device="cuda")
    return t


def _guard_intact(t, nbytes):
    tail = t[nbytes:].cpu().numpy()
    return bool(np.all(tail == CANARY)), int(np.count_nonzero(tail != CANARY))


@pytest.mark.parametrize("shape", [(37, 29, 23), (33, 17, 40), (61, 47, 35)])
def test_outputs_stay_inside_their_extent(S, shape):
    from paper_2112_10258_gb300 import capi
    vol = blob_volume(seed=11, shape=shape, n_blobs=24)
    nz, ny, nx = vol.shape
    d = torch.from_numpy(vol).cuda()
    st = torch.cuda.current_stream().cuda_stream
    det = S.Sift3D()

    # detect with room for everything, then with a capacity below the count
    _, n = det.detect(d, capacity=4096)
    assert n >= 2, "the volume must have keypoints"
    for cap in (n, n - 1, 1):
        out = _guarded(cap * 48)
        rc, need = capi.sift3d_detect(det.ctx, d.data_ptr(), 0, nx, ny, nz, st, out.data_ptr(), cap)
        torch.cuda.synchronize()
        assert need == n and rc in (capi.OK, capi.ECAPACITY)
        ok, bad = _guard_intact(out, cap * 48)
        assert ok, f"detect wrote {bad} guard bytes past capacity {cap}"

    # descriptors of exactly n keypoints (device count and host count)
    kps = _guarded(n * 48)
    rc, _ = capi.sift3d_detect(det.ctx, d.data_ptr(), 0, nx, ny, nz, st, kps.data_ptr(), n)
    assert rc == capi.OK
    for count in (n, -1):
        brief, rrief = _guarded(n * 8), _guarded(n * 64)
        assert capi.sift3d_describe(det.ctx, kps.data_ptr(), count, S.DESC_BOTH, brief.data_ptr(),
                                    rrief.data_ptr(), st) == capi.OK
        torch.cuda.synchronize()
        assert _guard_intact(brief, n * 8)[0] and _guard_intact(rrief, n * 64)[0], f"describe (n={count})"
    desc, rot = _guarded(n * 64), _guarded(n * 9 * 4)
    assert capi.sift3d_describe_siftrank(det.ctx, kps.data_ptr(), n, desc.data_ptr(), rot.data_ptr(), st) == capi.OK
    torch.cuda.synchronize()
    assert _guard_intact(desc, n * 64)[0] and _guard_intact(rot, n * 36)[0], "siftrank"

    # a pyramid level copied densely, and the standalone blur
    lvl = _guarded(nx * ny * nz * 4)
    assert capi.sift3d_read_level(det.ctx, 0, S.LEVEL_GAUSS, 2, lvl.data_ptr(), st) == capi.OK
    blur = _guarded(nx * ny * nz * 4)
    assert capi.sift3d_gaussian_blur(det.ctx, d.data_ptr(), nx, ny, nz, 1.7, blur.data_ptr(), st) == capi.OK
    torch.cuda.synchronize()
    assert _guard_intact(lvl, nx * ny * nz * 4)[0], "read_level"
    assert _guard_intact(blur, nx * ny * nz * 4)[0], "gaussian_blur"

    # matching of the descriptors against themselves
    for kind, rows in ((S.DESC_BRIEF, brief), (S.DESC_RRIEF, rrief)):
        nn, dist, dist2 = _guarded(n * 4), _guarded(n * 4), _guarded(n * 4)
        assert capi.sift3d_match(rows.data_ptr(), n, rows.data_ptr(), n, kind, nn.data_ptr(), dist.data_ptr(),
                                 dist2.data_ptr(), st) == capi.OK
        torch.cuda.synchronize()
        assert all(_guard_intact(t, n * 4)[0] for t in (nn, dist, dist2)), f"match kind {kind}"
    det.close()
