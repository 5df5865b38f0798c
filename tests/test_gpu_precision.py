"""Gaussian levels stored in FP16 / BF16 (arithmetic in FP32, DoG formed from
each level before rounding and stored in FP32): keypoint recall and precision
and descriptor agreement against the FP64 oracle on brain-like 145x174x145
volumes.  The 16-seed report is tests/precision_report.py; these tests hold
the floors on two seeds.

Floors.  FP16: the stated target, recall and precision >= 0.99.  Both
types: at least the recall and precision that the oracle's FP64 emulation of the
same storage arithmetic (build_pyramid_stored: levels rounded when stored,
residual-corrected DoG) reaches on the same volume, less 0.01 for the float32
arithmetic the device uses in place of float64.  The emulation runs on the CPU
and never sees a GPU result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sift3d_oracle as O  # noqa: E402
from tests.precision import descriptor_agreement, match_keypoints  # noqa: E402
from workloads.volumes import brain_like_volume  # noqa: E402

KINDS = {1: "f16", 2: "bf16"}


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    return S


@pytest.fixture(scope="module")
def refs():
    out = {}
    p = O.Params()
    for seed in (0, 1):
        vol = brain_like_volume(seed=seed)
        r = O.detect(vol, p)
        d = O.describe(r.pyramid, r.keypoints, p)
        emul = {}
        for kind in KINDS.values():
            e = O.detect_pyramid(O.build_pyramid_stored(vol, p, kind), p, keep_pyramid=False)
            _, rec, prec = match_keypoints(e.keypoints, r.keypoints)
            emul[kind] = (rec, prec)
        out[seed] = (vol, r, d, emul)
    return out


@pytest.mark.parametrize("storage,level_tol,min_bits", [(1, 2e-3, 0.97), (2, 1.5e-2, 0.90)])
def test_reduced_precision_storage(S, refs, storage, level_tol, min_bits):
    name = KINDS[storage]
    for seed, (vol, ref, dref, emul) in refs.items():
        det = S.Sift3D(storage=storage)
        buf, n = det.detect(torch.from_numpy(vol).cuda(), capacity=16384)
        kps = S.keypoints_to_numpy(buf, n)
        brief, rrief = det.describe(buf, n)
        b = brief[:n].cpu().numpy().view(np.uint64)
        r = rrief[: n * 64].cpu().numpy().reshape(n, 64)
        pairs, recall, precision = match_keypoints(kps, ref.keypoints)
        bits, ranks = descriptor_agreement(b, r, dref.brief, dref.rrief, pairs)
        g = det.read_level(0, S.LEVEL_GAUSS, 3, (145, 174, 145)).cpu().numpy()
        o = ref.pyramid.G[0][3]
        err = float(np.max(np.abs(g - o)) / np.max(np.abs(o)))
        e_rec, e_prec = emul[name]
        print(f"{name} seed {seed}: kp {n}/{ref.keypoints.size} recall {recall:.4f} precision {precision:.4f} "
              f"(emulation {e_rec:.4f} / {e_prec:.4f}) bits {bits:.4f} ranks {ranks:.4f} G3 err {err:.2e}")
        assert err <= level_tol
        assert recall >= e_rec - 0.01 and precision >= e_prec - 0.01
        if name == "f16":
            assert recall >= 0.99 and precision >= 0.99
        assert bits >= min_bits
        det.close()
