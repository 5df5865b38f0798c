"""FP64 CPU oracle of the 3D SIFT detector and the BRIEF / RRIEF descriptors.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The CUDA
library never calls it, and it shares no code with the CUDA path: both sides only
receive the same seeded input volumes from ``workloads/``.

Every function follows the paper (Carluer et al., "GPU optimization of the 3D
Scale-invariant Feature Transform Algorithm and a Novel BRIEF-inspired 3D Fast
Descriptor", arXiv 2112.10258) in plain numpy float64, step by step, with no
blocking or fusion:

* Gaussian scale space by recursive separable Gaussian filtering - Sec. 2 (Related
  Work, scale space generated recursively with separable 1D filters), Sec. 2.2.2
  "Gaussian Convolution" (three separable 1D convolutions in x, y, z), Fig. 8
  caption (6 convolutions per octave with increasing filter size).
* Sub-sampling by two: one output voxel from 8 input voxels - Sec. 2.2.2
  "Sub-sampling".
* Difference of Gaussians DoG(sigma) = I(sigma) - I(kappa sigma) - Sec. 2.2.2
  "Difference-of-Gaussian".
* 4D peak detection by the sum of signs over the 27+26+27 = 80 neighbours in three
  consecutive DoG volumes; peaks are +80, valleys -80, the cut is tunable - Sec.
  2.2.2 "4D Peak Detection" (sum-of-signs equation).  The extremum search here is
  the brute-force neighbour comparison the paper's CPU method uses (Sec. 4.4).
* BRIEF (binarised point-pair differences of a blurred patch) and RRIEF (the same
  differences, rank ordered) - Sec. 2.2.3; point-pair methods 1-5 (method 3,
  p1 ~ N(0, s), p2 ~ N(p1, s), by default); pre-blur sigma 0.95 (Sec. 4.5).
* Nearest-neighbour matching of descriptors - Sec. 2.1 (e).
* The 3D SIFT-Rank descriptor, the paper's comparison baseline, which the paper
  only outlines (Sec. 1: spherical gradient histogram orientation, 2x2x2 x 8
  bins, rank normalisation); the details are this implementation's reading.
* Sub-voxel refinement (one Newton step on the 4D DoG quadratic): not in the
  paper.
* Reduced-precision storage (not in the paper): ``build_pyramid_stored`` follows
  the same steps with the Gaussian levels rounded to 16 bits when stored and the
  DoG formed from each level's value before rounding; it predicts the recall of
  16-bit storage from the arithmetic alone.

Readings where the paper is silent:

* sigma0 = 1.6, sigma_in = 0.5, S = 3 scales per octave, S + 3 = 6 Gaussian levels
  with sigma_s = sigma0 * 2^(s/S); octave 0 starts with a blur of
  sqrt(sigma0^2 - sigma_in^2); level s is level s-1 blurred by
  sqrt(sigma_s^2 - sigma_{s-1}^2); octave o+1 starts from the sub-sample of level S.
* Discrete kernel w_k ~ exp(-k^2 / 2 sigma^2), |k| <= ceil(4 sigma), unit sum;
  clamp-to-edge boundary.
* DoG D_s = G_s - G_{s+1}; detection on D_1..D_S, interior voxels (border >= 1).
* Contrast test |D| >= t_c and a 3D Hessian curvature test (not in the paper).
* n = 64 point pairs, offsets in units of the keypoint's scale, clipped to
  |u|_inf <= 4 by resampling; pattern drawn with SplitMix64 + Box-Muller.

Arrays are numpy (nz, ny, nx), x fastest.

Parity bookkeeping: each decision of the detector is a comparison.  A comparison
whose FP64 margin is below ``REL_TOL`` x local magnitude is a *near tie*; the
oracle reports the voxels whose keypoint/non-keypoint outcome could flip under
such near ties (``DetectResult.uncertain``), so a float32 implementation may
differ from this oracle there and nowhere else.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

REL_TOL = 1e-5  # operand-margin tolerance relative to the local pyramid magnitude

KEYPOINT_DTYPE = np.dtype([
    ("octave", np.int32), ("scale", np.int32),
    ("ix", np.int32), ("iy", np.int32), ("iz", np.int32),
    ("polarity", np.int32), ("sign_sum", np.int32), ("dog", np.float64),
    ("x", np.float64), ("y", np.float64), ("z", np.float64), ("sigma", np.float64),
])


@dataclass
class Params:
    sigma0: float = 1.6
    sigma_in: float = 0.5
    scales_per_octave: int = 3
    min_octave_dim: int = 16
    max_octaves: int = 0          # 0 = until an octave would be smaller than min_octave_dim
    sign_sum_min: int = 80        # |sum of signs| cut; 80 = strict extremum
    border: int = 1
    contrast_thresh: float = 0.005
    curvature_r: float = 10.0
    trunc: float = 4.0
    desc_blur_sigma: float = 0.95
    desc_method: int = 3
    pattern_seed: int = 0x5EED5EED


# ----------------------------------------------------------------------------------
# Scale schedule (Sec. 2.2.2 Gaussian Convolution; Fig. 8 caption)
# ----------------------------------------------------------------------------------

def level_sigmas(p: Params) -> list[float]:
    """sigma_s = sigma0 * 2^(s/S) for the S+3 Gaussian levels of an octave."""
    S = p.scales_per_octave
    return [p.sigma0 * 2.0 ** (s / S) for s in range(S + 3)]


def initial_sigma(p: Params) -> float:
    """Blur that brings an input assumed at sigma_in up to sigma0."""
    return math.sqrt(p.sigma0 ** 2 - p.sigma_in ** 2)


def increment_sigmas(p: Params) -> list[float]:
    """Incremental blur from level s-1 to level s, s = 1..S+2."""
    sig = level_sigmas(p)
    return [math.sqrt(sig[s] ** 2 - sig[s - 1] ** 2) for s in range(1, len(sig))]


def octave_shapes(p: Params, shape_zyx) -> list[tuple[int, int, int]]:
    """Octave o has dims floor(dims / 2^o); keep octaves while min dim >= min_octave_dim."""
    shapes = []
    cur = tuple(int(v) for v in shape_zyx)
    while min(cur) >= p.min_octave_dim and (p.max_octaves <= 0 or len(shapes) < p.max_octaves):
        shapes.append(cur)
        cur = tuple(v // 2 for v in cur)
    return shapes


# ----------------------------------------------------------------------------------
# Gaussian convolution (Sec. 2.2.2: three separable 1D convolutions in x, y, z)
# ----------------------------------------------------------------------------------

def gaussian_radius(sigma: float, trunc: float = 4.0) -> int:
    return int(math.ceil(trunc * sigma))


def gaussian_taps(sigma: float, trunc: float = 4.0) -> np.ndarray:
    """Sampled Gaussian N(0, sigma^2) on k = -R..R, R = ceil(trunc*sigma), unit sum."""
    R = gaussian_radius(sigma, trunc)
    k = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def conv1d_clamp(vol: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """out[i] = sum_k taps[k] * vol[clamp(i + k - R)] along ``axis`` (edge replicate)."""
    R = (len(taps) - 1) // 2
    n = vol.shape[axis]
    idx = np.arange(n)
    out = np.zeros(vol.shape, np.float64)
    for j in range(len(taps)):
        src = np.clip(idx + (j - R), 0, n - 1)
        out += taps[j] * np.take(vol, src, axis=axis)
    return out


def blur3d(vol: np.ndarray, sigma: float, trunc: float = 4.0) -> np.ndarray:
    """Separable 3D Gaussian: an x pass, then a y pass, then a z pass."""
    taps = gaussian_taps(sigma, trunc)
    out = conv1d_clamp(np.asarray(vol, np.float64), taps, axis=2)
    out = conv1d_clamp(out, taps, axis=1)
    return conv1d_clamp(out, taps, axis=0)


# ----------------------------------------------------------------------------------
# Sub-sampling (Sec. 2.2.2: 8 input voxels give one output voxel)
# ----------------------------------------------------------------------------------

def subsample2(vol: np.ndarray) -> np.ndarray:
    """Mean of each 2x2x2 block; a trailing odd voxel on an axis is dropped."""
    Z, Y, X = (v // 2 for v in vol.shape)
    v = np.asarray(vol, np.float64)[: 2 * Z, : 2 * Y, : 2 * X]
    acc = np.zeros((Z, Y, X), np.float64)
    for a, b, c in itertools.product((0, 1), repeat=3):
        acc += v[a::2, b::2, c::2]
    return acc / 8.0


# ----------------------------------------------------------------------------------
# Pyramid: Gaussian levels and DoG (Sec. 2.2.2 "Difference-of-Gaussian")
# ----------------------------------------------------------------------------------

@dataclass
class Pyramid:
    G: list = field(default_factory=list)   # G[o][s], s = 0..S+2
    D: list = field(default_factory=list)   # D[o][s] = G[o][s] - G[o][s+1], s = 0..S+1


def input_to_float(vol: np.ndarray) -> np.ndarray:
    """float inputs are used as they are; uint8 codes map to [0, 1] by /255."""
    if vol.dtype == np.uint8:
        return vol.astype(np.float64) / 255.0
    return np.asarray(vol, np.float64)


def build_pyramid(vol: np.ndarray, p: Params) -> Pyramid:
    shapes = octave_shapes(p, vol.shape)
    incs = increment_sigmas(p)
    pyr = Pyramid()
    S = p.scales_per_octave
    for o in range(len(shapes)):
        if o == 0:
            g0 = blur3d(input_to_float(vol), initial_sigma(p), p.trunc)
        else:
            g0 = subsample2(pyr.G[o - 1][S])
        levels = [g0]
        for s in range(1, S + 3):
            levels.append(blur3d(levels[-1], incs[s - 1], p.trunc))
        pyr.G.append(levels)
        pyr.D.append([levels[s] - levels[s + 1] for s in range(S + 2)])
    return pyr


# ----------------------------------------------------------------------------------
# Reduced-precision storage (not in the paper): an FP64 emulation of the 16-bit
# storage scheme, from which the expected recall of FP16 / BF16 storage follows
# without the GPU.
# ----------------------------------------------------------------------------------

def round_to_storage(x: np.ndarray, kind: str) -> np.ndarray:
    """Round to the storage type and return float64: "f64" (unchanged), "f32",
    "f16" (IEEE half, round to nearest even), "bf16" (the upper 16 bits of the
    float32 value, round to nearest even)."""
    x = np.asarray(x, np.float64)
    if kind == "f64":
        return x
    if kind == "f32":
        return x.astype(np.float32).astype(np.float64)
    if kind == "f16":
        return x.astype(np.float16).astype(np.float64)
    if kind == "bf16":
        u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(kind)


def build_pyramid_stored(vol: np.ndarray, p: Params, kind: str) -> Pyramid:
    """The pyramid of build_pyramid with the Gaussian levels stored as ``kind``:
    every level is rounded when stored, the next level and the next octave's
    sub-sample are computed from the stored values, each level's rounding
    residual (value - stored value) is kept in IEEE half, and each DoG is
    D_{s-1} = (stored G_{s-1} + its residual) - G_s (G_s before rounding),
    stored in float32.  With kind "f64" this is build_pyramid exactly."""
    shapes = octave_shapes(p, vol.shape)
    incs = increment_sigmas(p)
    S = p.scales_per_octave
    exact = kind == "f64"
    pyr = Pyramid()
    for o in range(len(shapes)):
        if o == 0:
            g = blur3d(input_to_float(vol), initial_sigma(p), p.trunc)
        else:
            g = subsample2(pyr.G[o - 1][S])
        stored = round_to_storage(g, kind)
        res = g - stored if exact else round_to_storage(g - stored, "f16")
        levels, dogs = [stored], []
        for s in range(1, S + 3):
            gs = blur3d(levels[-1], incs[s - 1], p.trunc)
            d = (levels[-1] + res) - gs
            dogs.append(d if exact else round_to_storage(d, "f32"))
            stored = round_to_storage(gs, kind)
            res = gs - stored if exact else round_to_storage(gs - stored, "f16")
            levels.append(stored)
        pyr.G.append(levels)
        pyr.D.append(dogs)
    return pyr


# ----------------------------------------------------------------------------------
# 4D peak detection by sum of signs (Sec. 2.2.2 "4D Peak Detection"), contrast and
# curvature tests, and near-tie bookkeeping.
# ----------------------------------------------------------------------------------

NEIGHBOUR_OFFSETS = [d for d in itertools.product((-1, 0, 1), repeat=3)]  # (dz, dy, dx)


@dataclass
class DetectResult:
    keypoints: np.ndarray                       # KEYPOINT_DTYPE, canonical order
    uncertain: set = field(default_factory=set)  # {(o, s, iz, iy, ix)} with a near tie
    n_candidates: int = 0
    pyramid: Pyramid | None = None


def _robust(value: np.ndarray, bound: np.ndarray):
    """Decision value > 0 with first-order error ``bound``.
    Returns (robust_true, robust_false)."""
    return value > bound, value < -bound


def sum_of_signs(centre: np.ndarray, neighbours: list[np.ndarray]) -> np.ndarray:
    """f = sum over the neighbours of sign(D_centre - D_neighbour)."""
    S = np.zeros(centre.shape, np.int64)
    for nb in neighbours:
        S += np.sign(centre - nb).astype(np.int64)
    return S


def _hessian(Ds, cz, cy, cx):
    """Central-difference Hessian of D_s at the candidate voxels (entries of H)."""
    def d(dz, dy, dx):
        return Ds[cz + dz, cy + dy, cx + dx]
    c = d(0, 0, 0)
    hxx = d(0, 0, 1) + d(0, 0, -1) - 2.0 * c
    hyy = d(0, 1, 0) + d(0, -1, 0) - 2.0 * c
    hzz = d(1, 0, 0) + d(-1, 0, 0) - 2.0 * c
    hxy = (d(0, 1, 1) - d(0, -1, 1) - d(0, 1, -1) + d(0, -1, -1)) / 4.0
    hxz = (d(1, 0, 1) - d(-1, 0, 1) - d(1, 0, -1) + d(-1, 0, -1)) / 4.0
    hyz = (d(1, 1, 0) - d(-1, 1, 0) - d(1, -1, 0) + d(-1, -1, 0)) / 4.0
    return hxx, hyy, hzz, hxy, hxz, hyz


def curvature_test(h, polarity, r, eta=None):
    """Curvature test on H' = -polarity * H (a maximum has a negative definite H):
    H' positive definite by Sylvester's criterion (leading minors > 0) and
    tr(H')^3 * r^2 < (2r+1)^3 * det(H'), the 3D extension of the 2D edge test with
    eigenvalue ratio r (eigenvalues (a, ra, ra) give equality).

    With ``eta`` (per-DoG-value error allowance) also returns robust-true /
    robust-false masks from first-order error bounds of each quantity."""
    sgn = -polarity.astype(np.float64)
    a, b, c, xy, xz, yz = (sgn * v for v in h)
    m1 = a
    m2 = a * b - xy * xy
    det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz)
    tr = a + b + c
    k1 = (2.0 * r + 1.0) ** 3
    k2 = r * r
    g = k1 * det - k2 * tr ** 3
    ok = (m1 > 0) & (m2 > 0) & (det > 0) & (g > 0)
    if eta is None:
        return ok
    da = 4.0 * eta                     # |1| + |-2| + |1| DoG values per diagonal entry
    do = 1.0 * eta                     # 4 values x 1/4 per off-diagonal entry
    b_m1 = da
    b_m2 = np.abs(b) * da + np.abs(a) * da + 2.0 * np.abs(xy) * do
    cof_a = np.abs(b * c - yz * yz)
    cof_b = np.abs(a * c - xz * xz)
    cof_c = np.abs(a * b - xy * xy)
    cof_xy = 2.0 * np.abs(xy * c - yz * xz)
    cof_xz = 2.0 * np.abs(xy * yz - b * xz)
    cof_yz = 2.0 * np.abs(a * yz - xy * xz)
    b_det = (cof_a + cof_b + cof_c) * da + (cof_xy + cof_xz + cof_yz) * do
    b_g = k1 * b_det + 3.0 * k2 * tr * tr * (3.0 * da)
    parts = [(m1, b_m1), (m2, b_m2), (det, b_det), (g, b_g)]
    robust_true = np.ones(m1.shape, bool)
    robust_false = np.zeros(m1.shape, bool)
    for v, bd in parts:
        t, f = _robust(v, bd)
        robust_true &= t
        robust_false |= f
    return ok, robust_true, robust_false


def detect(vol: np.ndarray, p: Params, keep_pyramid: bool = True) -> DetectResult:
    return detect_pyramid(build_pyramid(vol, p), p, keep_pyramid)


def detect_pyramid(pyr: Pyramid, p: Params, keep_pyramid: bool = True) -> DetectResult:
    """Extrema of a built pyramid: the 80-neighbour sum of signs, the contrast
    and curvature tests, and the near-tie bookkeeping (Sec. 2.2.2)."""
    S = p.scales_per_octave
    sig = level_sigmas(p)
    rows = []
    uncertain = set()
    n_cand = 0
    for o in range(len(pyr.G)):
        G, D = pyr.G[o], pyr.D[o]
        Z, Y, X = D[0].shape
        b = p.border
        if Z < 2 * b + 1 or Y < 2 * b + 1 or X < 2 * b + 1:
            continue
        gmax = max(float(np.max(np.abs(g))) for g in G)
        tau_max = REL_TOL * gmax          # no local tolerance exceeds this
        T = p.sign_sum_min
        for s in range(1, S + 1):
            Ds = D[s]
            inner = Ds[b:Z - b, b:Y - b, b:X - b]
            # Necessary conditions, evaluated on every interior voxel: the contrast
            # test and the 26 neighbours in D_s, each counted as a near tie when
            # within tau_max.  A voxel that fails either even with every near tie
            # resolved in its favour can neither be a keypoint nor be uncertain.
            maybe = np.abs(inner) >= p.contrast_thresh - tau_max
            s26 = np.zeros(inner.shape, np.int16)
            n26 = np.zeros(inner.shape, np.int16)
            for dz, dy, dx in NEIGHBOUR_OFFSETS:
                if dz == 0 and dy == 0 and dx == 0:
                    continue
                nb = Ds[b + dz:Z - b + dz, b + dy:Y - b + dy, b + dx:X - b + dx]
                diff = inner - nb
                near = np.abs(diff) < tau_max
                s26 += np.where(near, 0, np.sign(diff)).astype(np.int16)
                n26 += near
            rest = 54
            maybe &= (s26 + n26 + rest >= T) | (s26 - n26 - rest <= -T)
            cz, cy, cx = np.nonzero(maybe)
            cz, cy, cx = cz + b, cy + b, cx + b
            if cz.size == 0:
                continue
            n_cand += cz.size
            c = Ds[cz, cy, cx]
            # local magnitude: largest |G| over the 3x3x3 neighbourhood in the four
            # Gaussian levels the three DoG volumes are formed from
            mag = np.zeros(c.shape)
            for lvl in range(s - 1, s + 3):
                for dz, dy, dx in NEIGHBOUR_OFFSETS:
                    mag = np.maximum(mag, np.abs(G[lvl][cz + dz, cy + dy, cx + dx]))
            tau = REL_TOL * mag
            # contrast |D| >= t_c
            con = np.abs(c) >= p.contrast_thresh
            con_rt = np.abs(c) - p.contrast_thresh >= tau
            con_rf = p.contrast_thresh - np.abs(c) > tau
            # sum of signs over the 80 neighbours (27 in D_{s-1}, 26 in D_s, 27 in D_{s+1})
            Ssum = np.zeros(c.shape, np.int64)
            S_rob = np.zeros(c.shape, np.int64)
            n_near = np.zeros(c.shape, np.int64)
            for lvl in (s - 1, s, s + 1):
                for dz, dy, dx in NEIGHBOUR_OFFSETS:
                    if lvl == s and dz == 0 and dy == 0 and dx == 0:
                        continue
                    diff = c - D[lvl][cz + dz, cy + dy, cx + dx]
                    sg = np.sign(diff).astype(np.int64)
                    near = np.abs(diff) < tau
                    Ssum += sg
                    S_rob += np.where(near, 0, sg)
                    n_near += near
            ext = np.abs(Ssum) >= T
            smax, smin = S_rob + n_near, S_rob - n_near
            ext_rt = (smin >= T) | (smax <= -T)
            ext_rf = (smax < T) & (smin > -T)
            polarity = np.where(Ssum > 0, 1, np.where(Ssum < 0, -1, 0))
            polarity = np.where(S_rob != 0, np.sign(S_rob), polarity).astype(np.int64)
            # curvature (Hessian) test on D_s, evaluated with the extremum's polarity
            h = _hessian(Ds, cz, cy, cx)
            cur, cur_rt, cur_rf = curvature_test(h, polarity, p.curvature_r, eta=tau / 2.0)
            keep = con & ext & cur
            rob_false = con_rf | ext_rf | cur_rf
            rob_true = con_rt & ext_rt & cur_rt
            unsure = ~rob_false & ~rob_true
            for i in np.nonzero(unsure)[0]:
                uncertain.add((o, s, int(cz[i]), int(cy[i]), int(cx[i])))
            for i in np.nonzero(keep)[0]:
                ix, iy, iz = int(cx[i]), int(cy[i]), int(cz[i])
                scale = 2.0 ** o
                rows.append((o, s, ix, iy, iz, int(polarity[i]), int(Ssum[i]), float(c[i]),
                             (ix + 0.5) * scale - 0.5, (iy + 0.5) * scale - 0.5,
                             (iz + 0.5) * scale - 0.5, sig[s] * scale))
    kps = np.array(rows, dtype=KEYPOINT_DTYPE)
    kps = sort_keypoints(kps)
    return DetectResult(kps, uncertain, n_cand, pyr if keep_pyramid else None)


def sort_keypoints(kps: np.ndarray) -> np.ndarray:
    """Canonical order (octave, scale, iz, iy, ix)."""
    if kps.size == 0:
        return kps
    order = np.lexsort((kps["ix"], kps["iy"], kps["iz"], kps["scale"], kps["octave"]))
    return kps[order]


# ----------------------------------------------------------------------------------
# Point-pair patterns (Sec. 2.2.3, methods 1-5) from SplitMix64 + Box-Muller
# ----------------------------------------------------------------------------------

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> tuple[int, int]:
    """One SplitMix64 step (Steele, Lea & Flood, OOPSLA 2014): returns (new_state, output)."""
    state = (state + SPLITMIX_GAMMA) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class NormalStream:
    """Standard normals: each draw takes two 53-bit uniforms u, v in (0, 1) and
    returns sqrt(-2 ln u) * cos(2 pi v) (Box & Muller, 1958)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def uniform(self) -> float:
        self.state, z = splitmix64(self.state)
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        u = self.uniform()
        v = self.uniform()
        return math.sqrt(-2.0 * math.log(u)) * math.cos(2.0 * math.pi * v)


N_PAIRS = 64
PATTERN_CLIP = 4.0


def pattern_method3(seed: int, n_pairs: int = N_PAIRS, clip: float = PATTERN_CLIP) -> np.ndarray:
    """Method 3: p1 ~ N(0, I), p2 ~ N(p1, I), in units of the keypoint scale; a point
    with any |coordinate| > clip is redrawn.  Returns (n_pairs, 2, 3) in (x, y, z)."""
    rng = NormalStream(seed)
    out = np.zeros((n_pairs, 2, 3))
    for k in range(n_pairs):
        while True:
            p1 = np.array([rng.normal() for _ in range(3)])
            if np.all(np.abs(p1) <= clip):
                break
        while True:
            p2 = p1 + np.array([rng.normal() for _ in range(3)])
            if np.all(np.abs(p2) <= clip):
                break
        out[k, 0], out[k, 1] = p1, p2
    return out


def _normal_point(rng: NormalStream, mean: np.ndarray, clip: float) -> np.ndarray:
    """mean + N(0, I), redrawn until every |coordinate| <= clip."""
    while True:
        q = mean + np.array([rng.normal() for _ in range(3)])
        if np.all(np.abs(q) <= clip):
            return q


def pattern_method1(seed: int, n_pairs: int = N_PAIRS, radius: float = 2.0) -> np.ndarray:
    """Method 1 (Sec. 2.2.3): p1 and p2 uniform in the ball of radius 2 sigma (the
    paper's 2D circle, in 3D), in units of the keypoint scale.  Each point is
    three uniforms on (-radius, radius) from the SplitMix64 stream, redrawn until
    it lies inside the ball.  Returns (n_pairs, 2, 3) in (x, y, z)."""
    rng = NormalStream(seed)

    def point():
        while True:
            q = np.array([radius * (2.0 * rng.uniform() - 1.0) for _ in range(3)])
            if q @ q <= radius * radius:
                return q

    out = np.zeros((n_pairs, 2, 3))
    for k in range(n_pairs):
        out[k, 0] = point()
        out[k, 1] = point()
    return out


def pattern_method2(seed: int, n_pairs: int = N_PAIRS, clip: float = PATTERN_CLIP) -> np.ndarray:
    """Method 2 (Sec. 2.2.3): p1 and p2 independent, each N(0, sigma) (keypoint-scale
    units); a point with any |coordinate| > clip is redrawn."""
    rng = NormalStream(seed)
    out = np.zeros((n_pairs, 2, 3))
    for k in range(n_pairs):
        out[k, 0] = _normal_point(rng, np.zeros(3), clip)
        out[k, 1] = _normal_point(rng, np.zeros(3), clip)
    return out


def pattern_method4(seed: int, n_pairs: int = N_PAIRS, clip: float = PATTERN_CLIP) -> np.ndarray:
    """Method 4 (Sec. 2.2.3, the paper's new method): p1 at the patch centre, p2 ~
    N(0, sigma) (keypoint-scale units), redrawn if any |coordinate| > clip."""
    rng = NormalStream(seed)
    out = np.zeros((n_pairs, 2, 3))
    for k in range(n_pairs):
        out[k, 1] = _normal_point(rng, np.zeros(3), clip)
    return out


POLAR_RADII = (0.5, 1.0, 1.5, 2.0)       # keypoint-scale units
POLAR_COS_THETA = (0.75, 0.25, -0.25, -0.75)


def pattern_method5(n_pairs: int = N_PAIRS) -> np.ndarray:
    """Method 5 (Sec. 2.2.3): p1 at the patch centre, p2 on a regular polar grid,
    read in 3D as spherical coordinates: 4 radii (0.5, 1, 1.5, 2 sigma) x 4 rings
    equally spaced in cos(theta) (0.75, 0.25, -0.25, -0.75) x 4 azimuths
    phi = pi/2 * a, rotated by pi/4 on odd rings.  Pair 16 m + 4 j + a has radius
    m, ring j, azimuth a.  Deterministic (no seed)."""
    out = np.zeros((n_pairs, 2, 3))
    for k in range(n_pairs):
        m, j, az = (k // 16) % 4, (k // 4) % 4, k % 4
        r, ct = POLAR_RADII[m], POLAR_COS_THETA[j]
        st = math.sqrt(1.0 - ct * ct)
        phi = 0.5 * math.pi * az + (0.25 * math.pi if j % 2 == 1 else 0.0)
        out[k, 1] = [r * st * math.cos(phi), r * st * math.sin(phi), r * ct]
    return out


def pattern_for(p: "Params") -> np.ndarray:
    """The point-pair pattern of p.desc_method (1..5) and p.pattern_seed."""
    if p.desc_method == 1:
        return pattern_method1(p.pattern_seed)
    if p.desc_method == 2:
        return pattern_method2(p.pattern_seed)
    if p.desc_method == 3:
        return pattern_method3(p.pattern_seed)
    if p.desc_method == 4:
        return pattern_method4(p.pattern_seed)
    if p.desc_method == 5:
        return pattern_method5()
    raise ValueError("desc_method must be 1..5")


# ----------------------------------------------------------------------------------
# Descriptors (Sec. 2.2.3): blur, sample point pairs, difference, binarise / rank
# ----------------------------------------------------------------------------------

def trilinear_clamp(V: np.ndarray, pts: np.ndarray):
    """Trilinear interpolation of V (Z, Y, X) at points (..., 3) given as (x, y, z)
    with each coordinate clamped to [0, dim-1].  Returns (values, max |corner|)."""
    Z, Y, X = V.shape
    px = np.clip(pts[..., 0], 0.0, X - 1.0)
    py = np.clip(pts[..., 1], 0.0, Y - 1.0)
    pz = np.clip(pts[..., 2], 0.0, Z - 1.0)
    x0, y0, z0 = (np.floor(q).astype(np.int64) for q in (px, py, pz))
    fx, fy, fz = px - x0, py - y0, pz - z0
    x1, y1, z1 = np.minimum(x0 + 1, X - 1), np.minimum(y0 + 1, Y - 1), np.minimum(z0 + 1, Z - 1)
    val = np.zeros(px.shape)
    mag = np.zeros(px.shape)
    for zi, wz in ((z0, 1.0 - fz), (z1, fz)):
        for yi, wy in ((y0, 1.0 - fy), (y1, fy)):
            for xi, wx in ((x0, 1.0 - fx), (x1, fx)):
                v = V[zi, yi, xi]
                val += wz * wy * wx * v
                mag = np.maximum(mag, np.abs(v))
    return val, mag


def rank_order(d: np.ndarray) -> np.ndarray:
    """Rank of each element, 0 = smallest; equal values ranked by lower index first."""
    n = d.shape[-1]
    ranks = np.zeros(d.shape, np.int64)
    for k in range(n):
        less = d < d[..., k:k + 1]
        equal_before = (d == d[..., k:k + 1]) & (np.arange(n) < k)
        ranks[..., k] = np.sum(less | equal_before, axis=-1)
    return ranks


@dataclass
class DescribeResult:
    brief: np.ndarray      # (n,) uint64, bit k = [d_k > 0]
    rrief: np.ndarray      # (n, 64) uint8 ranks
    d: np.ndarray          # (n, 64) float64 point-pair differences
    mag: np.ndarray        # (n, 64) local magnitude (largest |corner| of both samples)


def blurred_level(pyr: Pyramid, o: int, s: int, p: Params) -> np.ndarray:
    """The keypoint's Gaussian level G_s of octave o, pre-blurred by desc_blur_sigma."""
    if p.desc_blur_sigma <= 0.0:
        return pyr.G[o][s]
    return blur3d(pyr.G[o][s], p.desc_blur_sigma, p.trunc)


def describe(pyr: Pyramid, kps: np.ndarray, p: Params, pattern: np.ndarray | None = None,
             cache: dict | None = None) -> DescribeResult:
    if pattern is None:
        pattern = pattern_for(p)
    n = kps.size
    npair = pattern.shape[0]
    d = np.zeros((n, npair))
    mag = np.zeros((n, npair))
    sig = level_sigmas(p)
    cache = {} if cache is None else cache
    for i in range(n):
        o, s = int(kps["octave"][i]), int(kps["scale"][i])
        if (o, s) not in cache:
            cache[(o, s)] = blurred_level(pyr, o, s, p)
        B = cache[(o, s)]
        c = np.array([kps["ix"][i], kps["iy"][i], kps["iz"][i]], np.float64)
        p1 = c + sig[s] * pattern[:, 0, :]
        p2 = c + sig[s] * pattern[:, 1, :]
        v1, m1 = trilinear_clamp(B, p1)
        v2, m2 = trilinear_clamp(B, p2)
        d[i] = v1 - v2
        mag[i] = np.maximum(m1, m2)
    bits = (d > 0).astype(np.uint64)
    brief = np.zeros(n, np.uint64)
    for k in range(npair):
        brief |= bits[:, k] << np.uint64(k)
    rrief = rank_order(d).astype(np.uint8)
    return DescribeResult(brief, rrief, d, mag)


# ----------------------------------------------------------------------------------
# Matching (Sec. 2.1 (e)): nearest neighbour of each descriptor of A among B
# ----------------------------------------------------------------------------------

def hamming_distances(brief_a: np.ndarray, brief_b: np.ndarray) -> np.ndarray:
    """(na, nb) number of differing bits between the 64-bit BRIEF words."""
    x = brief_a.astype(np.uint64)[:, None] ^ brief_b.astype(np.uint64)[None, :]
    bits = (x[..., None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    return bits.sum(axis=-1).astype(np.int64)


def rank_distances(rrief_a: np.ndarray, rrief_b: np.ndarray) -> np.ndarray:
    """(na, nb) squared Euclidean distance between RRIEF rank vectors,
    sum_k (r_a[k] - r_b[k])^2."""
    a = rrief_a.astype(np.int64)
    b = rrief_b.astype(np.int64)
    return ((a[:, None, :] - b[None, :, :]) ** 2).sum(axis=-1)


def nearest_neighbours(dist: np.ndarray):
    """For each row: the index of the smallest distance (the lowest index among
    equal ones), that distance, and the smallest distance over the other
    columns (the second nearest; INT32_MAX if there is none).  An empty row set
    of columns gives index -1 and INT32_MAX distances."""
    na, nb = dist.shape
    big = 2 ** 31 - 1
    nn = np.full(na, -1, np.int64)
    d1 = np.full(na, big, np.int64)
    d2 = np.full(na, big, np.int64)
    for i in range(na):
        if nb == 0:
            continue
        j = int(np.argmin(dist[i]))          # first occurrence: lowest index
        nn[i], d1[i] = j, dist[i, j]
        if nb > 1:
            d2[i] = np.min(np.delete(dist[i], j))
    return nn, d1, d2


def match(desc_a: np.ndarray, desc_b: np.ndarray, kind: int):
    """kind 1 = BRIEF (uint64 words, Hamming distance), 2 = RRIEF ((n, 64) ranks,
    squared rank distance).  Returns nearest_neighbours of the distance matrix."""
    d = hamming_distances(desc_a, desc_b) if kind == 1 else rank_distances(desc_a, desc_b)
    return nearest_neighbours(d)


# ----------------------------------------------------------------------------------
# Sub-voxel refinement (no counterpart in the paper: the quadratic interpolation
# of Brown & Lowe, written for the 4D (x, y, z, scale) DoG stack)
# ----------------------------------------------------------------------------------

_REFINE_AXES = ((0, 0, 0, 1), (0, 0, 1, 0), (0, 1, 0, 0), (1, 0, 0, 0))   # x, y, z, level as (dl, dz, dy, dx)


def refine_derivatives(D: list, s: int, iz: int, iy: int, ix: int):
    """Centre value c, gradient g and Hessian H of the DoG stack at (ix, iy, iz)
    of level s, by central differences with unit steps in x, y, z and the level
    index (the usual 3-point first and second differences, and the 4-point
    mixed differences)."""
    def v(d):
        dl, dz, dy, dx = d
        return float(D[s + dl][iz + dz, iy + dy, ix + dx])

    def add(a, b, sa=1, sb=1):
        return tuple(sa * x + sb * y for x, y in zip(a, b))

    zero = (0, 0, 0, 0)
    c = v(zero)
    g = np.zeros(4)
    H = np.zeros((4, 4))
    for a, ea in enumerate(_REFINE_AXES):
        g[a] = 0.5 * (v(ea) - v(add(zero, ea, 1, -1)))
        H[a, a] = v(ea) + v(add(zero, ea, 1, -1)) - 2.0 * c
        for b in range(a + 1, 4):
            eb = _REFINE_AXES[b]
            H[a, b] = H[b, a] = 0.25 * (v(add(ea, eb)) - v(add(ea, eb, 1, -1)) - v(add(ea, eb, -1, 1))
                                        + v(add(ea, eb, -1, -1)))
    return c, g, H


def refine_offset(D: list, s: int, iz: int, iy: int, ix: int):
    """One Newton step on the 4D quadratic through the samples: offset =
    -H^-1 g in (x, y, z, level) units and the interpolated value
    c + g.offset / 2.  Returns (offset (4,), value, ok, cond(H)); ok is False
    (offset 0, value c) when H is singular to working precision."""
    c, g, H = refine_derivatives(D, s, iz, iy, ix)
    cond = float(np.linalg.cond(H)) if np.all(np.isfinite(H)) else np.inf
    if not cond < 1e12:
        return np.zeros(4), c, False, cond
    off = -np.linalg.solve(H, g)
    return off, c + 0.5 * float(g @ off), True, cond


def refine_keypoints(pyr: Pyramid, kps: np.ndarray, p: Params):
    """Refined (x, y, z, sigma) in input voxels and the interpolated DoG value of
    each keypoint: position ((i + offset) + 0.5) 2^o - 0.5 per axis, sigma
    sigma0 2^((s + offset_s) / S) 2^o.  Returns (offsets (n, 4), values (n,),
    coords (n, 4), ok (n,), cond (n,))."""
    S = p.scales_per_octave
    n = kps.size
    offs, vals, coords = np.zeros((n, 4)), np.zeros(n), np.zeros((n, 4))
    ok, cond = np.zeros(n, bool), np.zeros(n)
    for i in range(n):
        o, s = int(kps["octave"][i]), int(kps["scale"][i])
        ix, iy, iz = int(kps["ix"][i]), int(kps["iy"][i]), int(kps["iz"][i])
        offs[i], vals[i], ok[i], cond[i] = refine_offset(pyr.D[o], s, iz, iy, ix)
        scale = float(1 << o)
        coords[i, :3] = (np.array([ix, iy, iz], float) + offs[i, :3] + 0.5) * scale - 0.5
        coords[i, 3] = p.sigma0 * 2.0 ** ((s + offs[i, 3]) / S) * scale
    return offs, vals, coords, ok, cond


# ----------------------------------------------------------------------------------
# 3D SIFT-Rank descriptor (the paper's comparison baseline, Sec. 1 and Sec. 3.5:
# dominant orientation from peaks of a discrete spherical histogram of gradient,
# a 3x3 rotation; 2x2x2 spatial x 8 orientation bins = 64 elements after
# reorientation; rank normalisation).  The paper gives no further detail; the
# sampling grid, the 12-direction histogram and the octant binning below are
# this implementation's reading.
# ----------------------------------------------------------------------------------

SR_GRID = 8            # samples per axis of the cube [-r, r]^3, r = SR_RADIUS * sigma
SR_RADIUS = 3.0
SR_NEGLIGIBLE = 1e-5   # votes below this fraction of the largest bin do not count in the margins


def icosahedron_directions() -> np.ndarray:
    """The 12 unit vertices of the regular icosahedron: cyclic permutations of
    (0, +-1, +-phi), normalised; order: (0, a, b), (a, b, 0), (b, 0, a) with
    a, b running over +-1, +-phi."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    out = []
    for a in (1.0, -1.0):
        for b in (phi, -phi):
            out.append((0.0, a, b))
    for a in (1.0, -1.0):
        for b in (phi, -phi):
            out.append((a, b, 0.0))
    for a in (1.0, -1.0):
        for b in (phi, -phi):
            out.append((b, 0.0, a))
    v = np.array(out)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def siftrank_samples(sigma: float):
    """Sample offsets u (n, 3) and Gaussian weights w (n,): the SR_GRID^3 cell
    centres of [-r, r]^3, r = 3 sigma, that lie in the ball |u| <= r, weighted
    by exp(-|u|^2 / (2 (r/2)^2))."""
    r = SR_RADIUS * sigma
    t = ((np.arange(SR_GRID) + 0.5) / SR_GRID * 2.0 - 1.0) * r
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    u = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    keep = np.sum(u * u, axis=1) <= r * r
    u = u[keep]
    w = np.exp(-np.sum(u * u, axis=1) / (2.0 * (0.5 * r) ** 2))
    return u, w


def siftrank_gradients(G: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Gradient of G at points (n, 3) (x, y, z) by central differences of
    trilinear samples (coordinates clamped to the grid), unit steps."""
    g = np.zeros_like(pts)
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        vp, _ = trilinear_clamp(G, pts + e)
        vm, _ = trilinear_clamp(G, pts - e)
        g[:, a] = 0.5 * (vp - vm)
    return g


def siftrank_orientation(g: np.ndarray, w: np.ndarray):
    """Rotation R = [e1 e2 e3] (columns) from the gradients: e1 is the weighted
    mean gradient of the peak bin of the 12-direction histogram (each gradient
    votes w |g| into its nearest icosahedron direction); e2 is the same for the
    components perpendicular to e1, made exactly perpendicular; e3 = e1 x e2.
    Returns (R, margin): margin is the smallest of the relative gaps between
    each histogram's peak bin and its runner-up, and of the gaps between each
    vector's nearest and second-nearest direction (near-tie bookkeeping)."""
    V = icosahedron_directions()

    def peak(vec):
        mag = np.linalg.norm(vec, axis=1)
        dots = vec @ V.T
        b = np.argmax(dots, axis=1)
        hist = np.zeros(12)
        np.add.at(hist, b, w * mag)
        # nearest-vertex margin of the samples whose vote is not negligible
        # (a zero gradient, e.g. from clamped samples, votes nothing either way)
        # Exact ties between two directions come from exactly zero gradient
        # components (clamped samples at the border); they are decided the same
        # way (lowest index) in any precision, so only non-zero gaps count.
        big = w * mag > SR_NEGLIGIBLE * max(hist.max(), 1e-300)
        srt = np.sort(dots[big], axis=1)
        gaps = (srt[:, -1] - srt[:, -2]) / mag[big]
        gaps = gaps[gaps > 0.0]
        vgap = float(np.min(gaps)) if gaps.size else 1.0
        m = int(np.argmax(hist))
        top = np.sort(hist)[::-1]
        gap = (top[0] - top[1]) / max(top[0], 1e-300)
        mean = (w[b == m, None] * vec[b == m]).sum(axis=0)
        return mean, min(gap, vgap)

    m1, gap1 = peak(g)
    if not np.linalg.norm(m1) > 0.0:                  # no gradient at all: the identity frame
        return np.eye(3), 0.0
    e1 = m1 / np.linalg.norm(m1)
    gp = g - np.outer(g @ e1, e1)
    m2, gap2 = peak(gp)
    m2 = m2 - (m2 @ e1) * e1
    if not np.linalg.norm(m2) > 0.0:                  # no perpendicular gradient: any perpendicular axis
        m2 = np.cross(e1, [1.0, 0.0, 0.0] if abs(e1[0]) < 0.9 else [0.0, 1.0, 0.0])
        gap2 = 0.0
    e2 = m2 / np.linalg.norm(m2)
    e3 = np.cross(e1, e2)
    return np.stack([e1, e2, e3], axis=1), min(gap1, gap2)


def siftrank_descriptor(G: np.ndarray, c: np.ndarray, sigma: float):
    """64 rank-normalised gradient histogram of the keypoint at c (octave voxels)
    with scale sigma (octave voxels).  Samples at c + R u, gradients rotated into
    the keypoint frame (g' = R^T g); spatial bin = octant of u (x fastest),
    orientation bin = octant of g'; element 8 * spatial + orientation gets
    w |g'|.  Returns (ranks (64,), histogram (64,), R, decision margin)."""
    u, w = siftrank_samples(sigma)
    g0 = siftrank_gradients(G, c + u)
    R, gap = siftrank_orientation(g0, w)
    pts = c + u @ R.T
    g = siftrank_gradients(G, pts) @ R                  # g' = R^T g, row-wise
    sb = (u[:, 0] >= 0) + 2 * (u[:, 1] >= 0) + 4 * (u[:, 2] >= 0)
    ob = (g[:, 0] >= 0) + 2 * (g[:, 1] >= 0) + 4 * (g[:, 2] >= 0)
    hist = np.zeros(64)
    np.add.at(hist, 8 * sb + ob, w * np.linalg.norm(g, axis=1))
    nrm = np.linalg.norm(g, axis=1)
    big = w * nrm > SR_NEGLIGIBLE * max(hist.max(), 1e-300)          # octant decisions that matter
    edge = min(float(np.min(np.abs(g[big]) / nrm[big, None])) if big.any() else 1.0, gap)
    return rank_order(hist[None])[0].astype(np.uint8), hist, R, edge


def siftrank(pyr: Pyramid, kps: np.ndarray, p: Params):
    """SIFT-Rank descriptors of keypoints on their Gaussian level G_s (not
    pre-blurred).  Returns (ranks (n, 64) uint8, hists (n, 64), R (n, 3, 3),
    margins (n,))."""
    sig = level_sigmas(p)
    n = kps.size
    ranks = np.zeros((n, 64), np.uint8)
    hists = np.zeros((n, 64))
    rots = np.zeros((n, 3, 3))
    margins = np.zeros(n)
    for i in range(n):
        o, s = int(kps["octave"][i]), int(kps["scale"][i])
        c = np.array([kps["ix"][i], kps["iy"][i], kps["iz"][i]], np.float64)
        ranks[i], hists[i], rots[i], margins[i] = siftrank_descriptor(pyr.G[o][s], c, sig[s])
    return ranks, hists, rots, margins
