"""Sub-voxel refinement (params.refine): the GPU's float32 Newton step on the
4D DoG quadratic against the oracle's float64 step on the same keypoints, and
the keypoint set unchanged by it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sift3d_oracle as O  # noqa: E402
from workloads.volumes import blob_volume, brain_like_volume  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _detect(S, vol, **kw):
    det = S.Sift3D(**kw)
    buf, n = det.detect(torch.from_numpy(vol).cuda(), capacity=16384)
    kps = S.keypoints_to_numpy(buf, n)
    return det, kps


@pytest.mark.parametrize("which", ["blobs64", "brain145"])
def test_refinement_matches_oracle(S, which):
    """The offset is -H^-1 g from central differences of the DoG, so a sample
    error eps moves it by at most about ||H^-1|| eps (|dg| + |dH| |offset|) with
    |dg| <= eps and |dH| <= 4 eps per entry: the test bounds every keypoint by
    2 ||H^-1||_2 eps (2 + 8 |offset|), eps the measured largest difference
    between the GPU's and the oracle's DoG levels of that octave, and checks that
    the typical difference is far below it."""
    vol = blob_volume(seed=0) if which == "blobs64" else brain_like_volume(seed=2)
    det0, plain = _detect(S, vol)
    det0.close()
    det, ref = _detect(S, vol, refine=1)
    key = ("octave", "scale", "iz", "iy", "ix")
    assert plain.size == ref.size and all(np.array_equal(plain[f], ref[f]) for f in key)   # same set
    assert np.all(plain["refined"] == 0) and np.all(np.isin(ref["refined"], (1, 2)))

    p = O.Params()
    pyr = O.build_pyramid(vol, p)
    eps = []
    for o, D in enumerate(pyr.D):
        nz, ny, nx = D[0].shape
        eps.append(max(float(np.max(np.abs(det.read_level(o, S.LEVEL_DOG, s, (nx, ny, nz)).cpu().numpy() - D[s])))
                       for s in range(len(D))))
    det.close()
    kk = np.zeros(ref.size, O.KEYPOINT_DTYPE)
    for f in key:
        kk[f] = ref[f]
    offs, vals, coords, ok, cond = O.refine_keypoints(pyr, kk, p)
    scale = (1 << ref["octave"].astype(np.int64)).astype(np.float64)
    S_ = p.scales_per_octave
    got = np.zeros((ref.size, 4))
    got[:, 0] = (ref["x"] + 0.5) / scale - 0.5 - ref["ix"]
    got[:, 1] = (ref["y"] + 0.5) / scale - 0.5 - ref["iy"]
    got[:, 2] = (ref["z"] + 0.5) / scale - 0.5 - ref["iz"]
    got[:, 3] = np.log2(ref["sigma"] / (p.sigma0 * 2.0 ** (ref["scale"] / S_) * scale)) * S_
    bound = np.zeros(ref.size)
    for i in range(ref.size):
        _, _, H = O.refine_derivatives(pyr.D[int(ref["octave"][i])], int(ref["scale"][i]), int(ref["iz"][i]),
                                       int(ref["iy"][i]), int(ref["ix"][i]))
        hinv = 1.0 / max(np.linalg.svd(H, compute_uv=False).min(), 1e-300)
        bound[i] = 2.0 * hinv * eps[int(ref["octave"][i])] * (2.0 + 8.0 * np.linalg.norm(offs[i])) + 1e-6
    good = ok & (ref["refined"] == 1)
    assert good.mean() > 0.9
    diff = np.max(np.abs(got - offs), axis=1)
    print(which, "refined", int(good.sum()), "of", ref.size, "median |d offset|", float(np.median(diff[good])),
          "max |d offset|", float(diff[good].max()), "max diff/bound", float((diff[good] / bound[good]).max()),
          "median |offset|", float(np.median(np.abs(offs[good, :3]))), "DoG eps per octave", eps)
    assert np.all(diff[good] <= bound[good])
    assert np.median(diff[good]) < 1e-3
    # unrefined records (singular 4D Hessian) keep the voxel position
    bad = ref["refined"] == 2
    assert np.allclose(ref["x"][bad], (ref["ix"][bad] + 0.5) * scale[bad] - 0.5)
