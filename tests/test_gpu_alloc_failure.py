"""Allocation failures, injected on the host (sift3d_test_fail_allocation makes
the n-th device or pinned allocation report out-of-memory; no GPU fault): the
call that needed the memory returns SIFT3D_ENOMEM, frees what it had taken, and
the same context then works normally."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.volumes import blob_volume, brain_like_volume  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_detect_reports_enomem_then_recovers(S):
    from paper_2112_10258_gb300 import capi
    vol = blob_volume(seed=0)
    d = torch.from_numpy(vol).cuda()
    ref = S.Sift3D()
    buf_ref, n_ref = ref.detect(d, capacity=4096)
    want = S.keypoints_to_numpy(buf_ref, n_ref).tobytes()
    ref.close()
    free0 = _free_bytes()
    det = S.Sift3D()
    out = torch.empty(4096 * 48, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert capi.sift3d_test_fail_allocation(1) == capi.OK      # the arena allocation fails
    rc, _ = capi.sift3d_detect(det.ctx, d.data_ptr(), 0, 64, 64, 64, stream, out.data_ptr(), 4096)
    assert rc == capi.ENOMEM, rc
    rc, n = capi.sift3d_detect(det.ctx, d.data_ptr(), 0, 64, 64, 64, stream, out.data_ptr(), 4096)
    assert rc == capi.OK and n == n_ref
    assert S.keypoints_to_numpy(out, n).tobytes() == want
    det.close()
    assert _free_bytes() >= free0 - (32 << 20)


@pytest.mark.parametrize("nth", [1, 3, 6])
def test_served_request_reports_enomem_and_the_server_keeps_serving(S, nth):
    """The nth allocation of a new request's buffers (device workspace, device
    outputs or mapped pinned results) fails: that request ends with
    SIFT3D_ENOMEM, its partial buffers are freed, and the next requests of the
    same server are served with the usual results."""
    from paper_2112_10258_gb300 import capi
    vol = brain_like_volume(seed=11, shape=(72, 64, 60))
    free0 = _free_bytes()
    srv = S.Sift3D(max_inflight=2)
    assert capi.sift3d_test_fail_allocation(nth) == capi.OK
    t = srv.submit(vol)
    with pytest.raises(S.Sift3DError) as e:
        while srv.poll(t, 100000) is None:
            pass
    assert e.value.code == capi.ENOMEM
    assert capi.sift3d_test_fail_allocation(0) == capi.OK
    res = []
    for _ in range(2):
        t2 = srv.submit(vol)
        r = None
        while r is None:
            r = srv.poll(t2, 100000)
        assert r["status"] == 0 and r["n_keypoints"] > 0
        res.append(r["keypoints"].tobytes())
    assert res[0] == res[1]
    srv.close()
    assert _free_bytes() >= free0 - (32 << 20)
