"""Serving path (sift3d_submit / sift3d_poll) on the GPU: mixed sizes and dtypes
in flight at once, each result equal to the same volume detected and described
alone, admission under a small HBM budget, and error paths."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.volumes import blob_volume, brain_like_volume, to_uint8  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _alone(S, vol):
    det = S.Sift3D()
    d = torch.from_numpy(vol).cuda()
    buf, n = det.detect(d, capacity=8192)
    brief, rrief = det.describe(buf, n)
    out = (S.keypoints_to_numpy(buf, n), brief[:n].cpu().numpy().view(np.uint64),
           rrief[: n * 64].cpu().numpy().reshape(n, 64))
    det.close()
    return out


def _wait(srv, t, limit_s=60.0):
    t_end = time.monotonic() + limit_s
    while True:
        r = srv.poll(t, 100000)
        if r is not None:
            return r
        assert time.monotonic() < t_end, "request did not finish"


def test_mixed_stream_matches_alone(S):
    vols = [blob_volume(seed=1), brain_like_volume(seed=2, shape=(96, 80, 72)),
            to_uint8(brain_like_volume(seed=3, shape=(64, 70, 66))), blob_volume(seed=4, shape=(50, 60, 70)),
            brain_like_volume(seed=5)]
    alone = [_alone(S, v) for v in vols]
    srv = S.Sift3D(max_inflight=3, max_keypoints=8192)
    tickets = [srv.submit(v) for v in vols] + [srv.submit(v) for v in vols[::-1]]
    res = [_wait(srv, t) for t in tickets]
    for i, r in enumerate(res):
        k, b, rr = alone[i if i < len(vols) else 2 * len(vols) - 1 - i]
        assert r["status"] == 0
        assert r["n_keypoints"] == k.size == r["n_needed"]
        assert r["keypoints"].tobytes() == k.tobytes()
        assert np.array_equal(r["brief"], b) and np.array_equal(r["rrief"], rr)
        assert r["latency_ms"] >= r["queue_ms"] >= 0
    for t in tickets:
        assert srv.release(t) == 0
        assert srv.release(t) == -6  # ENOTFOUND after release
    srv.close()


def test_small_budget_serialises_but_completes(S):
    v = brain_like_volume(seed=7, shape=(96, 96, 96))
    from paper_2112_10258_gb300 import plan
    one = plan(96, 96, 96)["workspace_bytes"]
    srv = S.Sift3D(max_inflight=8, hbm_budget_bytes=int(one * 1.6) + (64 << 20))
    ts = [srv.submit(v) for _ in range(4)]
    res = [_wait(srv, t) for t in ts]
    assert all(r["status"] == 0 for r in res)
    assert len({r["keypoints"].tobytes() for r in res}) == 1
    srv.close()


def test_budget_too_small_is_rejected(S):
    srv = S.Sift3D(hbm_budget_bytes=1 << 20)
    with pytest.raises(S.Sift3DError) as e:
        srv.submit(blob_volume(seed=0))
    assert e.value.code == -7
    srv.close()


def test_capacity_reported_in_result(S):
    srv = S.Sift3D(max_keypoints=3)
    t = srv.submit(blob_volume(seed=0))
    r = _wait(srv, t)
    assert r["status"] == -3 and r["n_keypoints"] == 3 and r["n_needed"] > 3
    srv.close()


def test_device_resident_submit_matches_host_submit(S):
    """SIFT3D_SUBMIT_DEVICE: the request reads a CUDA volume in place (no
    host-to-device copy); results equal the host submit's, for float32 and uint8."""
    srv = S.Sift3D(max_inflight=2)
    for vol in (brain_like_volume(seed=8, shape=(80, 72, 64)), to_uint8(brain_like_volume(seed=9, shape=(64, 60, 56)))):
        host = _wait(srv, srv.submit(vol))
        d = torch.from_numpy(vol).cuda()
        dev = _wait(srv, srv.submit_device(d))
        assert host["status"] == dev["status"] == 0
        assert host["keypoints"].tobytes() == dev["keypoints"].tobytes()
        assert np.array_equal(host["brief"], dev["brief"]) and np.array_equal(host["rrief"], dev["rrief"])
    with pytest.raises(S.Sift3DError) as e:   # a host pointer is not device memory
        srv.submit_ptr(brain_like_volume(seed=8, shape=(16, 16, 16)).ctypes.data, S.DTYPE_F32, (16, 16, 16),
                       flags=S.SUBMIT_DEVICE)
    assert e.value.code == -1
    srv.close()
