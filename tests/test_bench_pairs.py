"""The similarity warp of `bench.py --mode pairs` (host code, no GPU): a
Gaussian bump at p in A peaks at T(p) in the warped volume, for translations,
rotations about z, scalings and their combination."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ndi = pytest.importorskip("scipy.ndimage")


def _bench():
    spec = importlib.util.spec_from_file_location("sift3d_bench_pairs", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("scale,deg,t", [(1.0, 0.0, (8, 16, 8)), (1.0, 30.0, (0, 0, 0)), (1.2, 0.0, (0, 0, 0)),
                                         (1.1, 20.0, (3, -2, 1))])
def test_warp_moves_a_bump_to_its_image(scale, deg, t):
    B = _bench()
    shape = (40, 50, 60)                      # (z, y, x)
    p = np.array([20.0, 30.0, 15.0])          # (x, y, z)
    A = np.zeros(shape)
    A[int(p[2]), int(p[1]), int(p[0])] = 1.0
    A = ndi.gaussian_filter(A, 2.0)
    forward, warp = B.similarity_transform(shape, scale, deg, t)
    W = warp(A)
    iz, iy, ix = np.unravel_index(np.argmax(W), W.shape)
    want = forward(p[None, :])[0]
    assert np.max(np.abs(np.array([ix, iy, iz]) - want)) <= 1.0, (want, (ix, iy, iz))
