"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test compares the oracle with something *other than itself*: a closed form,
a brute-force evaluation written differently (direct 3D sums, pure-Python loops,
eigenvalues instead of Sylvester minors), a library routine, or a published
reference sequence.  The mistakes these are chosen to catch: a dropped tap or a
wrong normalisation (unit sum, variance, ramp), wrong boundary handling (direct
3D clamp sum), a wrong sub-sampling phase (closed form), a wrong DoG sign or
scale (blob pin), a wrong neighbour set or tie rule (brute-force extrema), a
wrong curvature formula (eigenvalue check), and generator slips (published
vector).
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import sift3d_oracle as O
from workloads.volumes import blob_volume

# ------------------------------------------------------------------ Gaussian kernel


@pytest.mark.parametrize("sigma", [0.95, 1.2263, 1.5199, 1.9466, 2.4525, 3.09, 5.0])
def test_taps_unit_sum_symmetric_radius(sigma):
    w = O.gaussian_taps(sigma)
    R = (len(w) - 1) // 2
    assert R == math.ceil(4 * sigma)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.array_equal(w, w[::-1])
    assert np.all(np.diff(w[: R + 1]) > 0)  # increasing towards the centre


@pytest.mark.parametrize("sigma", [1.0, 1.5199, 2.4525, 3.09, 5.0])
def test_taps_discrete_variance_close_to_sigma_squared(sigma):
    w = O.gaussian_taps(sigma)
    R = (len(w) - 1) // 2
    k = np.arange(-R, R + 1)
    var = float(np.sum(k * k * w))
    # truncation at 4 sigma removes ~6e-5 of the mass in the tails
    assert abs(var / sigma ** 2 - 1.0) < 2e-3


def test_level_schedule_closed_form():
    p = O.Params()
    sig = O.level_sigmas(p)
    kappa = 2.0 ** (1.0 / 3.0)
    assert len(sig) == 6
    for s in range(1, 6):
        assert abs(sig[s] / sig[s - 1] - kappa) < 1e-14
    assert abs(sig[3] - 2 * p.sigma0) < 1e-14  # level S is twice sigma0: next octave base
    inc = O.increment_sigmas(p)
    for s in range(1, 6):
        assert abs(math.hypot(sig[s - 1], inc[s - 1]) - sig[s]) < 1e-14
    assert abs(math.hypot(O.initial_sigma(p), p.sigma_in) - p.sigma0) < 1e-14
    radii = [O.gaussian_radius(O.initial_sigma(p))] + [O.gaussian_radius(v) for v in inc]
    assert radii == [7, 5, 7, 8, 10, 13]


def test_octave_shapes():
    p = O.Params()
    assert O.octave_shapes(p, (145, 174, 145)) == [(145, 174, 145), (72, 87, 72), (36, 43, 36), (18, 21, 18)]
    assert O.octave_shapes(p, (64, 64, 64)) == [(64, 64, 64), (32, 32, 32), (16, 16, 16)]
    assert O.octave_shapes(p, (15, 64, 64)) == []
    assert O.octave_shapes(O.Params(max_octaves=2), (64, 64, 64)) == [(64, 64, 64), (32, 32, 32)]


# ------------------------------------------------------------------ separable convolution


def _direct_blur3d(vol, sigma):
    """Direct (non-separable) 3D sum with the outer-product kernel and clamped indices."""
    w = O.gaussian_taps(sigma)
    R = (len(w) - 1) // 2
    Z, Y, X = vol.shape
    zi, yi, xi = np.arange(Z), np.arange(Y), np.arange(X)
    out = np.zeros(vol.shape)
    for c in range(-R, R + 1):
        zz = np.clip(zi + c, 0, Z - 1)
        for b in range(-R, R + 1):
            yy = np.clip(yi + b, 0, Y - 1)
            plane = vol[np.ix_(zz, yy, np.arange(X))]
            wzy = w[c + R] * w[b + R]
            for a in range(-R, R + 1):
                xx = np.clip(xi + a, 0, X - 1)
                out += wzy * w[a + R] * plane[:, :, xx]
    return out


@pytest.mark.parametrize("sigma", [1.2263, 2.4525])
def test_separable_equals_direct_3d_convolution(sigma):
    rng = np.random.default_rng(1)
    vol = rng.standard_normal((16, 13, 11))  # R=10 exceeds half of every dim: clamp heavy
    assert np.max(np.abs(O.blur3d(vol, sigma) - _direct_blur3d(vol, sigma))) < 1e-12


def test_blur_preserves_constant_and_interior_ramp():
    const = np.full((12, 9, 10), 0.37)
    assert np.max(np.abs(O.blur3d(const, 2.0) - 0.37)) < 1e-15
    z, y, x = np.meshgrid(np.arange(30.), np.arange(28.), np.arange(26.), indexing="ij")
    ramp = 0.5 * x - 0.25 * y + 0.125 * z + 3.0
    out = O.blur3d(ramp, 1.5)  # R = 6
    R = 6
    inner = (slice(R, -R),) * 3
    assert np.max(np.abs(out[inner] - ramp[inner])) < 1e-12
    # at the clamped border the ramp is not preserved (edge replicate bends it)
    assert abs(out[0, 0, 0] - ramp[0, 0, 0]) > 1e-3


def test_blur_semigroup_in_interior():
    rng = np.random.default_rng(2)
    vol = rng.standard_normal((40, 40, 40))
    a, b = 1.5, 2.0
    two = O.blur3d(O.blur3d(vol, a), b)
    one = O.blur3d(vol, math.hypot(a, b))
    inner = (slice(12, -12),) * 3
    rel = np.max(np.abs(two[inner] - one[inner])) / np.max(np.abs(one[inner]))
    assert rel < 1e-3


# ------------------------------------------------------------------ sub-sampling


def test_subsample_closed_forms():
    assert np.all(O.subsample2(np.full((9, 8, 7), 2.5)) == 2.5)
    z, y, x = np.meshgrid(np.arange(9.), np.arange(8.), np.arange(7.), indexing="ij")
    out = O.subsample2(x + 10 * y + 100 * z)
    assert out.shape == (4, 4, 3)  # odd trailing voxel dropped
    K, J, I = np.meshgrid(np.arange(4.), np.arange(4.), np.arange(3.), indexing="ij")
    # block (2I, 2I+1) averages to 2I + 0.5 on every axis
    expect = (2 * I + 0.5) + 10 * (2 * J + 0.5) + 100 * (2 * K + 0.5)
    assert np.max(np.abs(out - expect)) < 1e-12


# ------------------------------------------------------------------ extrema and tests


def test_sum_of_signs_worked_examples():
    c = np.array([1.0])
    assert O.sum_of_signs(c, [np.array([0.0])] * 80)[0] == 80
    assert O.sum_of_signs(c, [np.array([0.0])] * 79 + [np.array([1.0])])[0] == 79   # tie: sign(0) = 0
    assert O.sum_of_signs(c, [np.array([0.0])] * 79 + [np.array([2.0])])[0] == 78
    assert O.sum_of_signs(-c, [np.array([0.0])] * 80)[0] == -80


def _brute_force_detect(vol, p):
    """Pure-Python detector on a tiny single-octave volume: explicit loops over
    voxels and the 80 neighbours, curvature by eigenvalues of the Hessian."""
    pyr = O.build_pyramid(vol, p)
    D = pyr.D[0]
    Z, Y, X = D[0].shape
    b = p.border
    out = set()
    r = p.curvature_r
    for s in range(1, p.scales_per_octave + 1):
        for z in range(b, Z - b):
            for y in range(b, Y - b):
                for x in range(b, X - b):
                    c = D[s][z, y, x]
                    if abs(c) < p.contrast_thresh:
                        continue
                    nbs = [D[l][z + dz, y + dy, x + dx] for l in (s - 1, s, s + 1)
                           for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                           if not (l == s and dz == 0 and dy == 0 and dx == 0)]
                    assert len(nbs) == 80
                    S = sum(1 for v in nbs if c > v) - sum(1 for v in nbs if c < v)
                    if abs(S) < p.sign_sum_min:
                        continue
                    pol = 1 if S > 0 else -1
                    Ds = D[s]
                    H = np.zeros((3, 3))
                    f = lambda dz, dy, dx: Ds[z + dz, y + dy, x + dx]
                    H[0, 0] = f(0, 0, 1) - 2 * c + f(0, 0, -1)
                    H[1, 1] = f(0, 1, 0) - 2 * c + f(0, -1, 0)
                    H[2, 2] = f(1, 0, 0) - 2 * c + f(-1, 0, 0)
                    H[0, 1] = H[1, 0] = (f(0, 1, 1) - f(0, 1, -1) - f(0, -1, 1) + f(0, -1, -1)) / 4
                    H[0, 2] = H[2, 0] = (f(1, 0, 1) - f(1, 0, -1) - f(-1, 0, 1) + f(-1, 0, -1)) / 4
                    H[1, 2] = H[2, 1] = (f(1, 1, 0) - f(1, -1, 0) - f(-1, 1, 0) + f(-1, -1, 0)) / 4
                    ev = np.linalg.eigvalsh(-pol * H)
                    if np.all(ev > 0) and ev.sum() ** 3 / np.prod(ev) < (2 * r + 1) ** 3 / r ** 2:
                        out.add((0, s, z, y, x))
    return out


def _grid_blob_volume(seed, shape=(26, 24, 22), spacing=9, sigma_range=(2.5, 3.5)):
    """Blobs on a jittered grid (so they stay separate) plus mild noise; sizes
    chosen so the scale-normalised response peaks on D_1..D_3 of octave 0."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = np.full((nz, ny, nx), 0.3)
    for cz in range(5, nz - 4, spacing):
        for cy in range(5, ny - 4, spacing):
            for cx in range(5, nx - 4, spacing):
                c = np.array([cx, cy, cz]) + rng.uniform(-1, 1, 3)
                sb = rng.uniform(*sigma_range)
                a = rng.choice([-1, 1]) * rng.uniform(0.3, 1.0)
                vol += a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * sb * sb))
    return vol + rng.normal(0, 0.01, vol.shape)


@pytest.mark.parametrize("seed,cut", [(0, 80), (1, 80), (2, 78)])
def test_detect_matches_brute_force_on_tiny_volumes(seed, cut):
    vol = _grid_blob_volume(seed)
    p = O.Params(min_octave_dim=16, max_octaves=1, contrast_thresh=0.01, sign_sum_min=cut)
    res = O.detect(vol, p)
    got = {(int(k["octave"]), int(k["scale"]), int(k["iz"]), int(k["iy"]), int(k["ix"]))
           for k in res.keypoints}
    ref = _brute_force_detect(vol, p)
    assert len(ref) >= 4
    assert (got ^ ref) <= res.uncertain
    assert len(got & ref) >= len(ref) - len(res.uncertain)


def test_sum_of_signs_equals_80_iff_strict_extremum_exhaustive():
    rng = np.random.default_rng(5)
    for trial in range(4):
        D = [rng.integers(0, 4, size=(6, 6, 6)).astype(np.float64) if trial % 2 else
             rng.standard_normal((6, 6, 6)) for _ in range(5)]   # integer levels force ties
        for s in (1, 2, 3):
            for z, y, x in itertools.product(range(1, 5), repeat=3):
                c = D[s][z, y, x]
                nbs = [D[l][z + dz, y + dy, x + dx] for l in (s - 1, s, s + 1)
                       for dz, dy, dx in O.NEIGHBOUR_OFFSETS if not (l == s and dz == dy == dx == 0)]
                S = int(O.sum_of_signs(np.array([c]), [np.array([v]) for v in nbs])[0])
                n_gt = sum(c > v for v in nbs)
                n_lt = sum(c < v for v in nbs)
                assert S == n_gt - n_lt
                assert (S == 80) == (c > max(nbs))
                assert (S == -80) == (c < min(nbs))


def test_detect_sign_sum_cut_admits_non_strict_extrema():
    vol = blob_volume(seed=3, shape=(20, 20, 20), n_blobs=10, sigma_range=(1.0, 2.5)).astype(np.float64)
    p80 = O.Params(min_octave_dim=16, max_octaves=1, contrast_thresh=0.001)
    p76 = O.Params(min_octave_dim=16, max_octaves=1, contrast_thresh=0.001, sign_sum_min=76)
    k80 = O.detect(vol, p80).keypoints
    k76 = O.detect(vol, p76).keypoints
    assert k76.size >= k80.size
    assert set(map(tuple, np.stack([k80["scale"], k80["iz"], k80["iy"], k80["ix"]], 1).tolist())) <= \
        set(map(tuple, np.stack([k76["scale"], k76["iz"], k76["iy"], k76["ix"]], 1).tolist()))
    assert np.all(np.abs(k80["sign_sum"]) == 80)
    assert np.all(np.abs(k76["sign_sum"]) >= 76)


def test_curvature_test_matches_eigenvalues():
    rng = np.random.default_rng(7)
    r = 10.0
    n_checked = 0
    for _ in range(4000):
        A = rng.standard_normal((3, 3))
        H = A @ A.T * rng.uniform(0.1, 2) - rng.uniform(0, 1) * np.eye(3)
        pol = rng.choice([-1, 1])
        Hn = -pol * H  # the test flips the sign for maxima
        h = tuple(np.array([v]) for v in (Hn[0, 0], Hn[1, 1], Hn[2, 2], Hn[0, 1], Hn[0, 2], Hn[1, 2]))
        ok = bool(O.curvature_test(h, np.array([-1]), r)[0])  # polarity -1 keeps the sign
        ev = np.linalg.eigvalsh(Hn)
        ref = bool(np.all(ev > 0) and ev.sum() ** 3 / np.prod(ev) < (2 * r + 1) ** 3 / r ** 2)
        assert ok == ref
        n_checked += ref
    assert n_checked > 100
    # boundary case: eigenvalues (a, r a, r a) give equality, so they are rejected
    h = tuple(np.array([v]) for v in (1.0, r, r, 0.0, 0.0, 0.0))
    assert not O.curvature_test(h, np.array([-1]), r)[0]
    h = tuple(np.array([v]) for v in (1.0, r * 0.99, r * 0.99, 0.0, 0.0, 0.0))
    assert O.curvature_test(h, np.array([-1]), r)[0]


def test_constant_volume_has_no_keypoints():
    res = O.detect(np.full((24, 20, 22), 0.4, np.float32), O.Params(contrast_thresh=0.0))
    assert res.keypoints.size == 0
    for levels in res.pyramid.D:
        for d in levels:
            assert np.max(np.abs(d)) < 1e-14


def _centred_blob(shape, centre_xyz, sigma_b, amp):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - centre_xyz[0]) ** 2 + (y - centre_xyz[1]) ** 2 + (z - centre_xyz[2]) ** 2
    return amp * np.exp(-r2 / (2 * sigma_b ** 2)) + 0.2


@pytest.mark.parametrize("sigma_b,octave", [(3.0, 0), (4.0, 0), (6.0, 1), (8.0, 1)])
@pytest.mark.parametrize("amp", [1.0, -1.0])
def test_blob_detected_at_centre_and_scale(sigma_b, octave, amp):
    """A Gaussian blob of std sigma_b maximises the scale-normalised 3D LoG at its
    centre at sigma = sigma_b * sqrt(2/3) (from s^2 lap L ~ s^2 / (sb^2 + s^2)^(5/2));
    the DoG keypoint must sit on the centre voxel of its octave, with the blob's
    polarity, within one scale step of that sigma."""
    f = 2 ** octave
    i = 32 // f
    c = (i + 0.5) * f - 0.5  # input coordinate of octave voxel i
    vol = _centred_blob((64, 64, 64), (c, c, c), sigma_b, amp)
    res = O.detect(vol, O.Params(contrast_thresh=0.001))
    k = res.keypoints
    hit = k[(k["ix"] == i) & (k["iy"] == i) & (k["iz"] == i) & (k["octave"] == octave)]
    assert hit.size == 1
    assert hit["polarity"][0] == (1 if amp > 0 else -1)
    assert abs(hit["x"][0] - c) < 1e-12 and abs(hit["z"][0] - c) < 1e-12
    target = sigma_b * math.sqrt(2.0 / 3.0)
    assert abs(math.log2(hit["sigma"][0] / target)) <= 1.0 / 3.0 + 1e-9
    # the strongest response of the volume is this keypoint
    assert np.argmax(np.abs(k["dog"])) == np.nonzero((k["ix"] == i) & (k["iy"] == i) & (k["iz"] == i)
                                                     & (k["octave"] == octave))[0][0]


def test_integer_shift_moves_every_keypoint():
    """Content away from the borders, shifted by 4 voxels (a multiple of 2^(O-1)
    for O = 3 octaves), moves every keypoint by exactly 4 input voxels."""
    core = _grid_blob_volume(21, shape=(36, 36, 36), spacing=10, sigma_range=(2.5, 4.5))
    base = np.full((80, 80, 80), 0.3)
    base[22:58, 22:58, 20:56] = core
    shift = 4
    moved = np.full_like(base, 0.3)
    moved[22:58, 22:58, 20 + shift:56 + shift] = core
    p = O.Params(contrast_thresh=0.005, max_octaves=3)
    r0, r1 = O.detect(base, p), O.detect(moved, p)
    k0, k1 = r0.keypoints, r1.keypoints
    assert k0.size > 5
    s0 = {(int(a), int(b), round(float(x) + shift, 6), round(float(y), 6), round(float(z), 6))
          for a, b, x, y, z in zip(k0["octave"], k0["scale"], k0["x"], k0["y"], k0["z"])}
    s1 = {(int(a), int(b), round(float(x), 6), round(float(y), 6), round(float(z), 6))
          for a, b, x, y, z in zip(k1["octave"], k1["scale"], k1["x"], k1["y"], k1["z"])}
    assert s0 == s1


# ------------------------------------------------------------------ pattern generator


def test_splitmix64_published_sequence(golden_dir):
    lines = [l for l in open(os.path.join(golden_dir, "splitmix64_seed1234567.txt")) if not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = [int(v) for v in lines[1:] if v.strip()]
    st, got = seed, []
    for _ in expect:
        st, z = O.splitmix64(st)
        got.append(z)
    assert got == expect


def test_normal_stream_moments():
    g = O.NormalStream(123)
    x = np.array([g.normal() for _ in range(40000)])
    assert abs(x.mean()) < 0.02
    assert abs(x.std() - 1.0) < 0.02
    assert abs(np.mean(x ** 3)) < 0.05
    assert abs(np.mean(x ** 4) - 3.0) < 0.1


def test_pattern_method3_properties():
    P = O.pattern_method3(0x5EED5EED)
    assert P.shape == (64, 2, 3)
    assert np.all(np.abs(P) <= 4.0)
    assert np.array_equal(P, O.pattern_method3(0x5EED5EED))
    assert not np.array_equal(P, O.pattern_method3(1))
    pts = np.concatenate([O.pattern_method3(sd) for sd in range(40)])
    p1, d = pts[:, 0, :], pts[:, 1, :] - pts[:, 0, :]
    assert abs(p1.mean()) < 0.06 and abs(p1.std() - 1.0) < 0.06         # p1 ~ N(0, 1)
    assert abs(d.mean()) < 0.06 and abs(d.std() - 1.0) < 0.08           # p2 ~ N(p1, 1)
    assert abs(np.corrcoef(p1.ravel(), d.ravel())[0, 1]) < 0.1


def test_pattern_method1_uniform_ball():
    P = O.pattern_method1(7)
    assert P.shape == (64, 2, 3)
    assert np.all(np.sum(P * P, axis=2) <= 4.0)                           # inside the radius-2 ball
    pts = np.concatenate([O.pattern_method1(sd).reshape(-1, 3) for sd in range(40)])
    r = np.sqrt(np.sum(pts * pts, axis=1))
    # uniform in a ball of radius R: P(r <= t) = (t/R)^3, E[r] = 3R/4, E[r^2] = 3R^2/5
    assert abs(r.mean() - 1.5) < 0.03 and abs(np.mean(r * r) - 2.4) < 0.06
    assert abs(np.mean(r <= 1.0) - 0.125) < 0.02
    assert abs(pts.mean()) < 0.05
    assert not np.array_equal(O.pattern_method1(7), O.pattern_method1(8))


def test_pattern_method2_independent_normals():
    pts = np.concatenate([O.pattern_method2(sd) for sd in range(40)])
    p1, p2 = pts[:, 0, :], pts[:, 1, :]
    assert np.all(np.abs(pts) <= 4.0)
    for q in (p1, p2):
        assert abs(q.mean()) < 0.06 and abs(q.std() - 1.0) < 0.06
    assert abs(np.corrcoef(p1.ravel(), p2.ravel())[0, 1]) < 0.1            # independent, unlike method 3


def test_pattern_method4_centre_and_normal():
    pts = np.concatenate([O.pattern_method4(sd) for sd in range(40)])
    assert np.all(pts[:, 0, :] == 0.0)                                     # p1 at the centre
    p2 = pts[:, 1, :]
    assert abs(p2.mean()) < 0.06 and abs(p2.std() - 1.0) < 0.06


def test_pattern_method5_polar_grid():
    P = O.pattern_method5()
    assert np.all(P[:, 0, :] == 0.0)
    r = np.sqrt(np.sum(P[:, 1, :] ** 2, axis=1))
    np.testing.assert_allclose(np.sort(np.unique(np.round(r, 12))), [0.5, 1.0, 1.5, 2.0], atol=1e-12)
    for m, rad in enumerate((0.5, 1.0, 1.5, 2.0)):
        np.testing.assert_allclose(r[16 * m: 16 * m + 16], rad, atol=1e-12)
    u = P[:16, 1, :] / 0.5                                                 # 16 distinct unit directions
    assert len({tuple(np.round(v, 9)) for v in u}) == 16
    np.testing.assert_allclose(u.sum(axis=0), 0.0, atol=1e-12)            # the grid is balanced
    np.testing.assert_allclose(np.sort(np.unique(np.round(u[:, 2], 12))), [-0.75, -0.25, 0.25, 0.75])


def test_pattern_for_dispatches_each_method():
    for m, fn in ((1, O.pattern_method1), (2, O.pattern_method2), (3, O.pattern_method3), (4, O.pattern_method4)):
        p = O.Params(desc_method=m, pattern_seed=99)
        np.testing.assert_array_equal(O.pattern_for(p), fn(99))
    np.testing.assert_array_equal(O.pattern_for(O.Params(desc_method=5)), O.pattern_method5())


# ------------------------------------------------------------------ descriptors


def test_trilinear_exact_for_linear_function_and_clamped():
    z, y, x = np.meshgrid(np.arange(7.), np.arange(6.), np.arange(5.), indexing="ij")
    V = 2 * x - 3 * y + 0.5 * z + 1
    pts = np.array([[1.25, 2.5, 3.75], [0, 0, 0], [4, 5, 6], [3.9, 0.1, 5.99]])
    val, mag = O.trilinear_clamp(V, pts)
    expect = 2 * pts[:, 0] - 3 * pts[:, 1] + 0.5 * pts[:, 2] + 1
    assert np.max(np.abs(val - expect)) < 1e-12
    out_of_range = np.array([[-3.0, 2.0, 1.0], [9.0, 2.0, 1.0]])
    val2, _ = O.trilinear_clamp(V, out_of_range)
    assert np.allclose(val2, [2 * 0 - 6 + 0.5 + 1, 2 * 4 - 6 + 0.5 + 1])


def test_rank_order_matches_stable_argsort():
    rng = np.random.default_rng(3)
    d = rng.integers(0, 10, size=(50, 64)).astype(float)   # many ties
    r = O.rank_order(d)
    ref = np.argsort(np.argsort(d, axis=1, kind="stable"), axis=1, kind="stable")
    assert np.array_equal(r, ref)
    for row in r:
        assert sorted(row.tolist()) == list(range(64))


def _tiny_keypoint(o, s, ix, iy, iz):
    k = np.zeros(1, O.KEYPOINT_DTYPE)
    k["octave"], k["scale"], k["ix"], k["iy"], k["iz"] = o, s, ix, iy, iz
    return k


def test_descriptor_hand_placed_pattern():
    """Pattern pair 0 = (centre, +1 sigma in x); pair 1 = (+0.5 sigma in y, centre).
    With no pre-blur the differences are plain trilinear reads of G."""
    p = O.Params(desc_blur_sigma=0.0, contrast_thresh=0.0)
    G = np.zeros((9, 9, 9))
    G[4, 4, 4] = 1.0
    G[4, 4, 6] = 3.0
    pyr = O.Pyramid(G=[[G] * 6], D=[])
    sig = O.level_sigmas(p)[1]  # 2.0159 octave voxels
    pattern = np.zeros((2, 2, 3))
    pattern[0, 1] = [1.0, 0.0, 0.0]
    pattern[1, 0] = [0.0, 0.5, 0.0]
    res = O.describe(pyr, _tiny_keypoint(0, 1, 4, 4, 4), p, pattern)
    # pair 0: G(c) - G(c + sig*x) = 1 - (value at x = 4 + 2.0159: between voxels 6 and 7)
    fx = 4 + sig - 6
    v = (1 - fx) * 3.0 + fx * 0.0
    assert abs(res.d[0, 0] - (1.0 - v)) < 1e-12
    # pair 1: y offset 1.008 -> weight (1 - 0.008) on voxel y=5 (zero), 0 at centre row
    assert abs(res.d[0, 1] - (0.0 - 1.0)) < 1e-12
    assert res.brief[0] == (1 if res.d[0, 0] > 0 else 0) | ((1 if res.d[0, 1] > 0 else 0) << 1)


def _random_keypoints(pyr, n, seed):
    """Keypoints at random octave/scale/positions, borders included (clamp paths)."""
    rng = np.random.default_rng(seed)
    k = np.zeros(n, O.KEYPOINT_DTYPE)
    for i in range(n):
        o = int(rng.integers(0, len(pyr.G)))
        Z, Y, X = pyr.G[o][0].shape
        k[i]["octave"], k[i]["scale"] = o, int(rng.integers(1, 4))
        k[i]["ix"], k[i]["iy"], k[i]["iz"] = rng.integers(0, X), rng.integers(0, Y), rng.integers(0, Z)
    return k


def _small_pyramid_and_kps(seed=4):
    vol = blob_volume(seed=seed, shape=(32, 30, 28), n_blobs=20, sigma_range=(1.0, 3.0), noise_std=0.01)
    p = O.Params(min_octave_dim=8, contrast_thresh=0.001)
    pyr = O.build_pyramid(vol, p)
    return vol, p, pyr, _random_keypoints(pyr, 40, seed)


def test_descriptor_affine_intensity_invariance_and_negation():
    vol, p, pyr, k = _small_pyramid_and_kps()
    d0 = O.describe(pyr, k, p)
    d2 = O.describe(O.build_pyramid(2.0 * vol.astype(np.float64) + 0.5, p), k, p)
    assert np.array_equal(d0.brief, d2.brief)
    assert np.array_equal(d0.rrief, d2.rrief)
    d3 = O.describe(O.build_pyramid(-vol.astype(np.float64), p), k, p)
    nz = d0.d != 0
    bits0 = (d0.brief[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    bits3 = (d3.brief[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    assert np.all((bits0 != bits3)[nz])
    assert np.array_equal(d3.rrief.astype(int), 63 - d0.rrief.astype(int))


def test_rrief_is_permutation_and_brief_bit_layout():
    vol, p, pyr, k = _small_pyramid_and_kps(seed=6)
    d = O.describe(pyr, k, p)
    for row in d.rrief:
        assert sorted(row.tolist()) == list(range(64))
    for i in range(d.d.shape[0]):
        for kbit in range(64):
            assert ((int(d.brief[i]) >> kbit) & 1) == int(d.d[i, kbit] > 0)


# ------------------------------------------------------------------ matching


def test_hamming_distance_counts_bits():
    rng = np.random.default_rng(3)
    a = rng.integers(0, 2 ** 63, 7, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 7, dtype=np.uint64)
    b = rng.integers(0, 2 ** 63, 5, dtype=np.uint64)
    D = O.hamming_distances(a, b)
    for i in range(7):
        for j in range(5):
            assert D[i, j] == bin(int(a[i]) ^ int(b[j])).count("1")
    assert O.hamming_distances(np.array([0], np.uint64), np.array([2 ** 64 - 1], np.uint64))[0, 0] == 64


def test_rank_distance_matches_spearman():
    # for permutations of 0..n-1: sum (a-b)^2 = n (n^2 - 1) / 6 * (1 - rho_spearman)
    from scipy.stats import spearmanr
    rng = np.random.default_rng(4)
    A = np.array([rng.permutation(64) for _ in range(6)], np.uint8)
    B = np.array([rng.permutation(64) for _ in range(4)], np.uint8)
    D = O.rank_distances(A, B)
    for i in range(6):
        for j in range(4):
            rho = spearmanr(A[i], B[j]).statistic
            assert abs(D[i, j] - 64 * (64 ** 2 - 1) / 6 * (1 - rho)) < 1e-6
    assert O.rank_distances(A[:1], A[:1])[0, 0] == 0
    assert O.rank_distances(np.arange(64, dtype=np.uint8)[None], np.arange(63, -1, -1, dtype=np.uint8)[None])[0, 0] \
        == 2 * 64 * (64 ** 2 - 1) // 6                                     # reversed order: rho = -1


def test_nearest_neighbours_ties_and_edges():
    D = np.array([[5, 3, 3, 9], [0, 0, 0, 0], [7, 8, 9, 1]])
    nn, d1, d2 = O.nearest_neighbours(D)
    assert nn.tolist() == [1, 0, 3] and d1.tolist() == [3, 0, 1] and d2.tolist() == [3, 0, 7]
    nn, d1, d2 = O.nearest_neighbours(np.zeros((2, 1), np.int64))
    assert nn.tolist() == [0, 0] and d2.tolist() == [2 ** 31 - 1] * 2
    nn, d1, d2 = O.nearest_neighbours(np.zeros((3, 0), np.int64))
    assert nn.tolist() == [-1] * 3 and d1.tolist() == [2 ** 31 - 1] * 3
    # a descriptor set matched against itself finds itself at distance 0
    rng = np.random.default_rng(5)
    W = rng.integers(0, 2 ** 63, 20, dtype=np.uint64)
    nn, d1, _ = O.match(W, W, 1)
    assert nn.tolist() == list(range(20)) and not d1.any()


# ------------------------------------------------------------------ sub-voxel refinement


def _quadratic_stack(centre, H, g0, c0, shape=(7, 7, 7), levels=5):
    """D_l(z, y, x) = c0 + g0.u + u.H.u / 2 with u = (x, y, z, l) - centre."""
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    out = []
    for l in range(levels):
        u = np.stack([x - centre[0], y - centre[1], z - centre[2], np.full_like(x, l - centre[3])], axis=-1)
        out.append(c0 + u @ g0 + 0.5 * np.einsum("...i,ij,...j->...", u, H, u))
    return out


def test_refinement_recovers_the_extremum_of_a_quadratic():
    # central differences are exact for a quadratic, so one Newton step lands
    # on its extremum: offset = true extremum - sample point
    rng = np.random.default_rng(2)
    A = rng.normal(size=(4, 4))
    H = -(A @ A.T + 4 * np.eye(4))                  # negative definite: a maximum
    ext = np.array([3.3, 2.8, 3.1, 2.2])             # extremum in (x, y, z, level)
    D = _quadratic_stack(ext, H, np.zeros(4), 0.7)
    off, val, ok, cond = O.refine_offset(D, 2, 3, 3, 3)
    assert ok
    np.testing.assert_allclose(off, ext - np.array([3, 3, 3, 2]), atol=1e-9)
    assert abs(val - 0.7) < 1e-9                     # the value at the extremum


def test_refinement_of_an_exact_sample_point_is_zero_and_singular_is_flagged():
    H = -np.diag([1.0, 2.0, 3.0, 0.5])
    D = _quadratic_stack(np.array([3.0, 3.0, 3.0, 2.0]), H, np.zeros(4), -0.2)
    off, val, ok, _ = O.refine_offset(D, 2, 3, 3, 3)
    assert ok and np.allclose(off, 0.0) and abs(val + 0.2) < 1e-12
    flat = [np.zeros((7, 7, 7)) for _ in range(5)]
    off, val, ok, cond = O.refine_offset(flat, 2, 3, 3, 3)
    assert not ok and not off.any()


# ------------------------------------------------------------------ 3D SIFT-Rank


def test_icosahedron_directions():
    V = O.icosahedron_directions()
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    D = V @ V.T
    off = D[~np.eye(12, dtype=bool)]
    # every other vertex is at dot +-1/sqrt(5), except the antipode at -1
    assert np.all((np.abs(np.abs(off) - 1 / np.sqrt(5)) < 1e-12) | (np.abs(off + 1) < 1e-12))
    assert np.all(np.sum(np.abs(D - 1 / np.sqrt(5)) < 1e-12, axis=1) == 5)   # five nearest neighbours each


def test_siftrank_samples_exact_enumeration():
    # cell centre i of the 8-cell axis is u = (2i - 7) / 8 in units of r, so it
    # lies in the ball |u| <= 1 iff sum (2i - 7)^2 <= 64: an integer count
    cells = [(i, j, k) for k in range(8) for j in range(8) for i in range(8)
             if (2 * i - 7) ** 2 + (2 * j - 7) ** 2 + (2 * k - 7) ** 2 <= 64]
    sigma = 1.7
    r = 3.0 * sigma
    u, w = O.siftrank_samples(sigma)
    assert len(cells) == u.shape[0] == w.shape[0] == 280
    expect = np.array([[(2 * i - 7) / 8.0, (2 * j - 7) / 8.0, (2 * k - 7) / 8.0] for i, j, k in cells]) * r
    np.testing.assert_allclose(u, expect, rtol=0, atol=1e-12)          # same points, same (z, y, x) order
    q = np.array([(2 * i - 7) ** 2 + (2 * j - 7) ** 2 + (2 * k - 7) ** 2 for i, j, k in cells]) / 64.0
    np.testing.assert_allclose(w, np.exp(-q / (2 * 0.5 ** 2)), rtol=1e-14)   # exp(-|u|^2 / (2 (r/2)^2))
    # every spatial octant (sign pattern) holds 35 samples, and each axis
    # reflection maps the set onto itself
    octant = (u[:, 0] >= 0) + 2 * (u[:, 1] >= 0) + 4 * (u[:, 2] >= 0)
    assert np.bincount(octant, minlength=8).tolist() == [35] * 8
    key = {tuple(np.round(p / r * 8).astype(int)) for p in u}
    for axis in range(3):
        flip = np.ones(3)
        flip[axis] = -1
        assert {tuple(np.round(p * flip / r * 8).astype(int)) for p in u} == key


def _analytic_volume(fn, shape=(40, 40, 40)):
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    return fn(x, y, z)


def test_siftrank_orientation_follows_the_dominant_gradient():
    G = _analytic_volume(lambda x, y, z: 2.0 * x + 0.5 * np.sin(0.7 * y) + 0.05 * np.cos(0.3 * z))
    ranks, hist, R, margin = O.siftrank_descriptor(G, np.array([20.0, 20.0, 20.0]), 2.0)
    assert abs(R[:, 0] @ [1, 0, 0]) > 0.99                  # e1 along the dominant x gradient
    assert abs(R[:, 1] @ [0, 1, 0]) > 0.95                  # e2 along the next (y) structure
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
    assert np.linalg.det(R) > 0
    assert sorted(ranks.tolist()) == list(range(64))


def test_siftrank_invariances():
    G = _analytic_volume(lambda x, y, z: np.sin(0.3 * x + 0.1 * y) * np.cos(0.25 * z - 0.2 * y) + 0.1 * x)
    c = np.array([19.0, 21.0, 18.0])
    r0, h0, R0, _ = O.siftrank_descriptor(G, c, 2.2)
    r1, h1, R1, _ = O.siftrank_descriptor(3.0 * G + 7.0, c, 2.2)           # affine intensity
    np.testing.assert_array_equal(r0, r1)
    np.testing.assert_allclose(R0, R1, atol=1e-9)
    Gs = np.roll(G, (2, -3, 4), axis=(0, 1, 2))                               # integer translation
    r2, _, R2, _ = O.siftrank_descriptor(Gs, c + np.array([4.0, -3.0, 2.0]), 2.2)
    np.testing.assert_array_equal(r0, r2)
    # I -> -I: e1, e2 flip and e3 stays, so the spatial x, y bits and the
    # orientation z bit of every element flip: a fixed permutation of the bins
    r3, h3, R3, _ = O.siftrank_descriptor(-G, c, 2.2)
    np.testing.assert_allclose(R3, R0 * np.array([-1.0, -1.0, 1.0]), atol=1e-9)
    perm = np.array([8 * ((k // 8) ^ 3) + ((k % 8) ^ 4) for k in range(64)])
    np.testing.assert_allclose(h3[perm], h0, rtol=1e-9)


# ---- reduced-precision storage emulation (not in the paper) -------------------

def test_round_to_storage_matches_the_formats():
    """bf16 keeps the upper 16 bits of the float32 value with round to nearest,
    ties to even (8 significant bits: relative error at most 2^-8); f16 is IEEE
    half (2^-11); f32 is float32 (2^-24)."""
    one = 1.0
    cases = [(one + 2 ** -8, one),                    # halfway, even neighbour below
             (one + 3 * 2 ** -8, one + 2 ** -6),      # halfway, even neighbour above
             (one + 2 ** -8 + 2 ** -20, one + 2 ** -7),   # just above halfway
             (-(one + 3 * 2 ** -8), -(one + 2 ** -6)), (0.0, 0.0), (3.0, 3.0)]
    for x, want in cases:
        assert O.round_to_storage(np.array([x]), "bf16")[0] == want, x
    rng = np.random.default_rng(3)
    x = rng.uniform(-2.0, 2.0, 10000)
    for kind, eps in (("bf16", 2.0 ** -8), ("f16", 2.0 ** -11), ("f32", 2.0 ** -24)):
        r = O.round_to_storage(x, kind)
        assert np.all(np.abs(r - x) <= eps * np.abs(x) * (1 + 1e-12) + (2.0 ** -25 if kind == "f16" else 0.0))
    assert np.array_equal(O.round_to_storage(x, "f16"), x.astype(np.float16).astype(np.float64))
    assert np.array_equal(O.round_to_storage(x, "f64"), x)


def test_stored_pyramid_emulation():
    """Without rounding the emulation is build_pyramid exactly; with 16-bit
    storage the Gaussian levels are representable in the format, and the DoG,
    formed from the levels before rounding, is far closer to the FP64 DoG than
    the stored levels are to the FP64 levels."""
    vol = blob_volume(seed=2, shape=(36, 34, 32), n_blobs=10)
    p = O.Params(min_octave_dim=16)
    ref = O.build_pyramid(vol, p)
    same = O.build_pyramid_stored(vol, p, "f64")
    for a, b in zip(ref.G + ref.D, same.G + same.D):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for kind in ("f16", "bf16"):
        st = O.build_pyramid_stored(vol, p, kind)
        for o in range(len(ref.G)):
            gmax = max(float(np.max(np.abs(g))) for g in ref.G[o])
            for g in st.G[o]:
                assert np.array_equal(O.round_to_storage(g, kind), g)
            g_err = max(float(np.max(np.abs(a - b))) for a, b in zip(st.G[o], ref.G[o]))
            d_err = max(float(np.max(np.abs(a - b))) for a, b in zip(st.D[o], ref.D[o]))
            unit = 2.0 ** (-8 if kind == "bf16" else -11)
            assert g_err <= 4 * unit * gmax
            assert d_err < 0.5 * g_err, (kind, o, d_err, g_err)
