"""Per-stage timing (sift3d_stage_times) switched on by params.profile or by the
SIFT3D_PROFILE environment variable, read at context creation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.volumes import blob_volume  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _stage_rows(S, det, vol):
    from paper_2112_10258_gb300 import capi
    det.detect(torch.from_numpy(vol).cuda(), capacity=4096)
    return capi.sift3d_stage_times(det.ctx)


def test_profile_from_environment(S, monkeypatch):
    vol = blob_volume(seed=2, shape=(48, 40, 36), n_blobs=10)
    monkeypatch.delenv("SIFT3D_PROFILE", raising=False)
    det = S.Sift3D()
    rc, rows = _stage_rows(S, det, vol)
    assert rc != 0 and rows == []            # not profiled
    det.close()
    monkeypatch.setenv("SIFT3D_PROFILE", "1")
    det = S.Sift3D()
    rc, rows = _stage_rows(S, det, vol)
    det.close()
    assert rc == 0 and len(rows) > 0
    labels = [r[0] for r in rows]
    assert any(".peak" in l for l in labels) and labels[-1] == "sort"
    assert all(np.isfinite(r[1]) and r[1] >= 0.0 for r in rows)
