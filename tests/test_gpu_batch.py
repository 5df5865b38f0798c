"""Batched detect + describe (sift3d_detect_batch): volumes of uneven sizes
under one graph launch, every pass a persistent launch over all volumes' tiles.
Each volume's keypoints, BRIEF words and RRIEF ranks must equal the
single-volume path bit for bit, with one wave and with a budget that forces
several waves, for float32 and uint8 input."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.volumes import brain_like_volume, to_uint8  # noqa: E402

SHAPES = [(96, 110, 100), (160, 130, 120), (64, 64, 64), (200, 120, 96), (120, 200, 140), (100, 96, 180)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _single(S, d, capacity, **kw):
    det = S.Sift3D(**kw)
    buf, n = det.detect(d, capacity=capacity)
    brief, rrief = det.describe(buf, n)
    out = (S.keypoints_to_numpy(buf, n).tobytes(), brief[:n].cpu().numpy().tobytes(),
           rrief[: n * 64].cpu().numpy().tobytes())
    det.close()
    return out


@pytest.mark.parametrize("budget_gib,u8", [(40, False), (1, False), (40, True)])
def test_batch_equals_single_volume_path(S, budget_gib, u8):
    vols = [brain_like_volume(seed=30 + i, shape=s) for i, s in enumerate(SHAPES)]
    if u8:
        vols = [to_uint8(v) for v in vols]
    dev = [torch.from_numpy(v).cuda() for v in vols]
    cap = 8192
    want = [_single(S, d, cap) for d in dev]
    det = S.Sift3D(hbm_budget_bytes=budget_gib << 30)
    for rep in range(2):   # the second call replays the cached graph
        res = det.detect_batch(dev, capacity=cap)
        torch.cuda.synchronize()
        for i, (buf, n, brief, rrief) in enumerate(res):
            got = (S.keypoints_to_numpy(buf, n).tobytes(), brief[:n].cpu().numpy().tobytes(),
                   rrief[: n * 64].cpu().numpy().tobytes())
            assert n > 0 and got == want[i], f"volume {i} {SHAPES[i]} (call {rep})"
    det.close()


def test_batch_separate_preblur_equals_single_volume_path(S):
    """A descriptor pre-blur of radius 5 (sigma 1.2) cannot ride on the level
    passes, so the batch runs it as separate passes."""
    vols = [brain_like_volume(seed=50 + i, shape=s) for i, s in enumerate(SHAPES[:3])]
    dev = [torch.from_numpy(v).cuda() for v in vols]
    cap = 8192
    want = [_single(S, d, cap, desc_blur_sigma=1.2) for d in dev]
    det = S.Sift3D(desc_blur_sigma=1.2)
    res = det.detect_batch(dev, capacity=cap)
    torch.cuda.synchronize()
    for i, (buf, n, brief, rrief) in enumerate(res):
        got = (S.keypoints_to_numpy(buf, n).tobytes(), brief[:n].cpu().numpy().tobytes(),
               rrief[: n * 64].cpu().numpy().tobytes())
        assert n > 0 and got == want[i], f"volume {i} {SHAPES[i]}"
    det.close()


def test_batch_rejects_unsupported_configurations(S):
    det = S.Sift3D(storage=S.STORAGE_F16)
    d = torch.zeros((20, 20, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(S.Sift3DError) as e:
        det.detect_batch([d])
    assert e.value.code == -1
    det.close()
