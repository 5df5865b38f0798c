"""Nearest-neighbour matching on the GPU (sift3d_match) against the oracle's
brute-force definition, and on a synthetic volume pair related by a known
translation (the paper's OASIS pairs are not available)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sift3d_oracle as O  # noqa: E402
from workloads.volumes import brain_like_volume  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


def _gpu_match(S, a, b, kind):
    ta = torch.from_numpy(a.view(np.int64) if kind == 1 else a).cuda()
    tb = torch.from_numpy(b.view(np.int64) if kind == 1 else b).cuda()
    nn, d1, d2 = S.match(ta, tb, kind)
    return nn.cpu().numpy(), d1.cpu().numpy(), d2.cpu().numpy()


def _check(got, ref):
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g.astype(np.int64), r)


@pytest.mark.parametrize("na,nb", [(300, 517), (1, 1), (33, 2), (64, 1000)])
def test_brief_matching_equals_oracle(S, na, nb):
    rng = np.random.default_rng(na * 7 + nb)
    b = rng.integers(0, 2 ** 63, nb, dtype=np.uint64) ^ (rng.integers(0, 2, nb, dtype=np.uint64) << np.uint64(63))
    a = rng.integers(0, 2 ** 63, na, dtype=np.uint64)
    a[: na // 3] = b[rng.integers(0, nb, na // 3)]                        # exact hits
    if nb > 4:
        b[1::4] = b[0::4][: len(b[1::4])]                                  # duplicate candidates: ties
    _check(_gpu_match(S, a, b, 1), O.match(a, b, 1))


@pytest.mark.parametrize("na,nb", [(200, 333), (1, 1), (40, 2)])
def test_rrief_matching_equals_oracle(S, na, nb):
    rng = np.random.default_rng(na + 13 * nb)
    b = np.array([rng.permutation(64) for _ in range(nb)], np.uint8)
    a = np.array([rng.permutation(64) for _ in range(na)], np.uint8)
    a[: na // 4] = b[rng.integers(0, nb, na // 4)]
    if nb > 4:
        b[2::5] = b[0::5][: len(b[2::5])]
    _check(_gpu_match(S, a, b, 2), O.match(a, b, 2))


def test_rank_distance_is_general_for_any_bytes(S):
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, (50, 64), dtype=np.uint8)
    b = rng.integers(0, 256, (70, 64), dtype=np.uint8)
    _check(_gpu_match(S, a, b, 2), O.match(a, b, 2))


def test_matching_edge_cases(S):
    a = np.arange(5, dtype=np.uint64)
    nn, d1, d2 = _gpu_match(S, a, np.zeros(0, np.uint64), 1)
    assert nn.tolist() == [-1] * 5 and d1.tolist() == [2 ** 31 - 1] * 5 and d2.tolist() == [2 ** 31 - 1] * 5
    nn, d1, d2 = _gpu_match(S, a, np.array([3], np.uint64), 1)
    assert nn.tolist() == [0] * 5 and d2.tolist() == [2 ** 31 - 1] * 5
    from paper_2112_10258_gb300 import capi
    assert capi.sift3d_match(0, 0, 0, 0, 1, 0, 0, 0, 0) == capi.OK                # nothing to do
    assert capi.sift3d_match(0, 3, 0, 0, 7, 0, 0, 0, 0) == capi.EINVAL             # bad kind


def test_synthetic_pair_matching_inliers(S):
    """Two crops of one brain-like volume, offset by (8, 16, 8) voxels in (x, y, z)
    (a multiple of 2^3, so every octave's grid shifts by whole voxels), the
    second with its own N(0, 0.01) noise.  A match is an inlier when the matched
    keypoints have the same octave and scale and their positions differ by the
    offset within one octave voxel.  Inlier counts are printed for BRIEF and
    RRIEF; the nearest neighbours of the GPU are checked against the oracle's
    on a sample of queries."""
    V = brain_like_volume(seed=3)
    sx, sy, sz = 8, 16, 8
    nz, ny, nx = V.shape
    A = np.ascontiguousarray(V[: nz - sz, : ny - sy, : nx - sx])
    rng = np.random.default_rng(11)
    B = np.ascontiguousarray(V[sz:, sy:, sx:] + rng.normal(0, 0.01, A.shape).astype(np.float32))
    res = []
    for vol in (A, B):
        det = S.Sift3D()
        buf, n = det.detect(torch.from_numpy(vol).cuda(), capacity=16384)
        kps = S.keypoints_to_numpy(buf, n)
        brief, rrief = det.describe(buf, n)
        sr = det.describe_siftrank(buf, n)
        res.append((kps, brief[:n].clone(), rrief[: n * 64].clone().view(n, 64), sr[: n * 64].clone().view(n, 64)))
        det.close()
    (ka, ba, ra, sa), (kb, bb, rb, sb) = res
    assert ka.size > 200 and kb.size > 200
    report = {}
    for kind, da, db in ((1, ba, bb), (2, ra, rb), (3, sa, sb)):
        name = kind
        kind = min(kind, 2)                 # SIFT-Rank ranks use the rank distance
        nn, d1, d2 = (t.cpu().numpy() for t in S.match(da, db, kind))
        sel = np.arange(0, ka.size, max(1, ka.size // 60))
        ref = O.match((da.cpu().numpy().view(np.uint64) if kind == 1 else da.cpu().numpy())[sel],
                      db.cpu().numpy().view(np.uint64) if kind == 1 else db.cpu().numpy(), kind)
        _check((nn[sel], d1[sel], d2[sel]), ref)
        m = kb[nn]
        scale = (1 << ka["octave"].astype(np.int64)).astype(np.float64)
        same = (m["octave"] == ka["octave"]) & (m["scale"] == ka["scale"])
        dx = (ka["x"] - sx) - m["x"]
        dy = (ka["y"] - sy) - m["y"]
        dz = (ka["z"] - sz) - m["z"]
        close = np.maximum(np.abs(dx), np.maximum(np.abs(dy), np.abs(dz))) <= scale
        ratio = d1 < 0.8 * d2
        report[name] = (int(np.sum(same & close)), int(np.sum(same & close & ratio)), int(np.sum(ratio)), ka.size)
    print("inliers (all NN, ratio-test NN, ratio-test matches, queries): BRIEF", report[1], "RRIEF", report[2],
          "SIFT-Rank", report[3])
    for kind in (1, 2, 3):
        inl, inl_r, n_r, nq = report[kind]
        assert inl >= 0.3 * nq                     # most shifted keypoints find their twin
        assert inl_r >= 0.8 * n_r                  # the ratio test keeps mostly inliers
