"""Pins of the oracle's near-tie bookkeeping (``DetectResult.uncertain``).

Every parity test excuses a GPU/oracle keypoint difference only where the oracle
flags the voxel as a near tie, so the flagged set itself must be right:

* sound: a perturbation of every DoG value by less than half the tolerance
  (1e-5 x the local pyramid magnitude, the per-comparison margin of the
  tolerance rule) flips a voxel's keypoint outcome only if the voxel is flagged;
* tight: every flagged voxel really is within reach of a flip, i.e. a
  perturbation of at most ``C_TIGHT`` times that allowance flips it.

The decisions are recomputed here from their definitions (Sec. 2.2.2 "4D Peak
Detection": the sum of signs over the 80 neighbours; the contrast cut; the
curvature test by the eigenvalues of the negated Hessian), not through the
oracle's vectorised detect, and the tolerance is this file's own constant, so a
change of the oracle's ``REL_TOL`` or of its error bounds shows up here.
"""
import itertools

import numpy as np
import pytest

from oracle import sift3d_oracle as O
from workloads.volumes import blob_volume, brain_like_volume

REL = 1e-5                 # the comparison tolerance (relative to the local magnitude)
# A voxel flagged for a near comparison or a near contrast cut must flip under
# C_TIGHT times the allowance: those margins are exact, and the allowance of the
# two values of a comparison adds up to 0.7-1.0 of the tolerance.  A voxel
# flagged only by the curvature test may need C_TIGHT_CURV: that test's error
# bounds are first order and add per-entry maxima over the six Hessian entries,
# while the three diagonal entries share the centre value (a change of it moves
# them together), which overstates the reachable change up to about 2x; and the
# bound takes half the tolerance per value where the allowance is 0.3-0.5 of it.
C_TIGHT = 2.0
C_TIGHT_CURV = 4.0
OFFS = list(itertools.product((-1, 0, 1), repeat=3))   # (dz, dy, dx)


# ---------------------------------------------------------------------------
# decisions from their definitions
# ---------------------------------------------------------------------------

def _curvature_ok(Hs, polarity, r):
    """H' = -polarity * H positive definite and tr(H')^3 r^2 < (2r+1)^3 det(H'),
    evaluated through the eigenvalues of each 3x3 matrix."""
    Hp = -polarity[:, None, None] * Hs
    lam = np.linalg.eigvalsh(Hp)
    det = np.prod(lam, axis=1)
    tr = np.sum(lam, axis=1)
    return np.all(lam > 0, axis=1) & ((2 * r + 1) ** 3 * det - r * r * tr ** 3 > 0)


def _hessians(Ds, z, y, x):
    """Central-difference Hessians of D_s at the given voxels, shape (n, 3, 3) (x, y, z)."""
    def v(dz, dy, dx):
        return Ds[z + dz, y + dy, x + dx]
    c = v(0, 0, 0)
    H = np.empty((len(z), 3, 3))
    H[:, 0, 0] = v(0, 0, 1) + v(0, 0, -1) - 2 * c
    H[:, 1, 1] = v(0, 1, 0) + v(0, -1, 0) - 2 * c
    H[:, 2, 2] = v(1, 0, 0) + v(-1, 0, 0) - 2 * c
    H[:, 0, 1] = H[:, 1, 0] = (v(0, 1, 1) - v(0, -1, 1) - v(0, 1, -1) + v(0, -1, -1)) / 4
    H[:, 0, 2] = H[:, 2, 0] = (v(1, 0, 1) - v(-1, 0, 1) - v(1, 0, -1) + v(-1, 0, -1)) / 4
    H[:, 1, 2] = H[:, 2, 1] = (v(1, 1, 0) - v(-1, 1, 0) - v(1, -1, 0) + v(-1, -1, 0)) / 4
    return H


def _octave_keypoints(D, S, p):
    """{(s, z, y, x): polarity} of one octave from its DoG levels D[0..S+1]."""
    out = {}
    b = p.border
    Z, Y, X = D[0].shape
    if min(Z, Y, X) < 2 * b + 1:
        return out
    for s in range(1, S + 1):
        c = D[s][b:Z - b, b:Y - b, b:X - b]
        ssum = np.zeros(c.shape, np.int64)
        for lvl in (s - 1, s, s + 1):
            for dz, dy, dx in OFFS:
                if lvl == s and (dz, dy, dx) == (0, 0, 0):
                    continue
                ssum += np.sign(c - D[lvl][b + dz:Z - b + dz, b + dy:Y - b + dy, b + dx:X - b + dx]).astype(np.int64)
        cand = (np.abs(c) >= p.contrast_thresh) & (np.abs(ssum) >= p.sign_sum_min)
        z, y, x = np.nonzero(cand)
        if z.size == 0:
            continue
        pol = np.sign(ssum[z, y, x])
        z, y, x = z + b, y + b, x + b
        ok = _curvature_ok(_hessians(D[s], z, y, x), pol, p.curvature_r)
        for i in np.nonzero(ok)[0]:
            out[(s, int(z[i]), int(y[i]), int(x[i]))] = int(pol[i])
    return out


def _value_allowance(G, rel):
    """Largest perturbation of each DoG value D_l(v) that keeps every comparison it
    enters within the tolerance rule: D_l = G_l - G_{l+1}, and every stencil
    using D_l(v) takes its local magnitude over both levels at v, so
    rel/2 * max(|G_l(v)|, |G_{l+1}(v)|) is below half of each such tolerance."""
    return [0.5 * rel * np.maximum(np.abs(G[l]), np.abs(G[l + 1])) for l in range(len(G) - 1)]


def _volumes():
    blobs = blob_volume(seed=0)                                  # 64^3, 40 blobs
    brain = brain_like_volume(seed=0)
    nz, ny, nx = brain.shape
    crop = np.ascontiguousarray(brain[nz // 4: nz // 4 + 72, ny // 4: ny // 4 + 87, nx // 4: nx // 4 + 72])
    return {"blobs64": blobs, "brain_crop72x87x72": crop}


@pytest.fixture(scope="module")
def detected():
    p = O.Params()
    return {name: (vol, O.detect(vol, p)) for name, vol in _volumes().items()}, p


# ---------------------------------------------------------------------------
# soundness
# ---------------------------------------------------------------------------

def test_recomputed_decisions_equal_the_oracle_keypoints(detected):
    """The decision functions of this file reproduce the oracle's keypoint set
    (so the perturbation tests below compare like with like)."""
    res, p = detected
    S = p.scales_per_octave
    for name, (vol, r) in res.items():
        got = set()
        for o, D in enumerate(r.pyramid.D):
            got |= {(o,) + k for k in _octave_keypoints(D, S, p)}
        want = {(int(k["octave"]), int(k["scale"]), int(k["iz"]), int(k["iy"]), int(k["ix"])) for k in r.keypoints}
        assert got == want, name


@pytest.mark.parametrize("rel_scale", [1.0, 30.0])
def test_flips_under_allowed_perturbation_are_flagged(detected, monkeypatch, rel_scale):
    """Random perturbations of every DoG value within the allowance (uniform, and
    at the corners of the allowance box) flip only flagged voxels.  At 30x the
    tolerance (the oracle recomputed with the same scale) flips are frequent, so
    the bookkeeping logic is exercised on many voxels, not only on the few near
    ties of the production tolerance."""
    res, p = detected
    S = p.scales_per_octave
    rel = REL * rel_scale
    n_flips = 0
    for name, (vol, r0) in res.items():
        if rel_scale != 1.0:
            monkeypatch.setattr(O, "REL_TOL", rel)
            r = O.detect(vol, p)
            monkeypatch.setattr(O, "REL_TOL", REL)
        else:
            r = r0
        for o, (G, D) in enumerate(zip(r.pyramid.G, r.pyramid.D)):
            base = _octave_keypoints(D, S, p)
            allow = _value_allowance(G, rel)
            for trial in range(6):
                rng = np.random.default_rng(1000 * o + trial)
                if trial % 2 == 0:
                    u = [rng.uniform(-1.0, 1.0, size=d.shape) for d in D]
                else:   # corners of the box, just inside
                    u = [np.where(rng.random(d.shape) < 0.5, -0.999, 0.999) for d in D]
                Dp = [d + a * e for d, a, e in zip(D, allow, u)]
                pert = _octave_keypoints(Dp, S, p)
                flips = {k for k in set(base) | set(pert) if base.get(k) != pert.get(k)}
                n_flips += len(flips)
                unflagged = {(o,) + k for k in flips} - r.uncertain
                assert not unflagged, f"{name}: flips outside the flagged set: {sorted(unflagged)[:5]}"
    if rel_scale > 1.0:
        assert n_flips >= 20, f"only {n_flips} flips: the test did not exercise the bookkeeping"


# ---------------------------------------------------------------------------
# tightness
# ---------------------------------------------------------------------------

def _local(Dlist, s, z, y, x):
    """The 3x3x3 neighbourhoods of D_{s-1}, D_s, D_{s+1} around (z, y, x): (3, 3, 3, 3)."""
    return np.stack([Dlist[l][z - 1:z + 2, y - 1:y + 2, x - 1:x + 2] for l in (s - 1, s, s + 1)]).astype(np.float64)


def _local_tests(L, p):
    """(contrast passed, |sum of signs| >= cut, curvature passed, polarity) of the
    centre of a local stencil (3, 3, 3, 3) of D_{s-1}, D_s, D_{s+1}."""
    c = L[1, 1, 1, 1]
    d = np.delete(c - L.reshape(-1), 40)      # 40: the centre itself
    ssum = int(np.sum(np.sign(d)))
    pol = int(np.sign(ssum)) or 1
    H = _hessians(L[1], np.array([1]), np.array([1]), np.array([1]))
    curv = bool(_curvature_ok(H, np.array([pol]), p.curvature_r)[0])
    return abs(c) >= p.contrast_thresh, abs(ssum) >= p.sign_sum_min, curv, pol


def _local_decision(L, p):
    """Keypoint outcome and polarity of the centre of a local stencil."""
    con, ext, curv, pol = _local_tests(L, p)
    return con and ext and curv, pol


def _flip_directions(L, p):
    """Candidate unit perturbation fields (entries in [-1, 1]) of a stencil that
    aim to flip its outcome: toward the contrast cut and away from it; each
    comparison closed (centre and neighbour move toward each other) or opened;
    the gradient sign of each curvature quantity, both ways; all failing
    comparisons of a polarity fixed at once."""
    dirs = []
    c = L[1, 1, 1, 1]
    e_c = np.zeros_like(L)
    e_c[1, 1, 1, 1] = 1.0
    dirs += [e_c, -e_c]
    flat = L.reshape(-1)
    for k in range(81):
        if k == 40:
            continue
        e = np.zeros(81)
        sg = np.sign(c - flat[k]) or 1.0
        e[k], e[40] = sg, -sg            # close comparison k
        dirs += [e.reshape(L.shape), -e.reshape(L.shape)]
    for pol in (1, -1):                  # resolve every comparison in favour of one polarity
        e = np.zeros(81)
        for k in range(81):
            if k != 40 and pol * (c - flat[k]) <= 0:
                e[k] = -pol
        e[40] = pol
        dirs.append(e.reshape(L.shape))
    # curvature quantities: leading minors, det and the edge test, by finite differences
    def quantities(Lx, pol):
        H = -pol * _hessians(Lx[1], np.array([1]), np.array([1]), np.array([1]))[0]
        r = p.curvature_r
        return np.array([H[0, 0], H[0, 0] * H[1, 1] - H[0, 1] ** 2, np.linalg.det(H),
                         (2 * r + 1) ** 3 * np.linalg.det(H) - r * r * np.trace(H) ** 3])
    for pol in (1, -1):
        q0 = quantities(L, pol)
        h = 1e-7 * max(1e-12, np.max(np.abs(L)))
        grad = np.zeros((4,) + L.shape)
        for idx in itertools.product(range(3), repeat=3):
            Lp = L.copy()
            Lp[(1,) + idx] += h
            grad[(slice(None), 1) + idx] = (quantities(Lp, pol) - q0) / h
        for j in range(4):
            g = np.sign(grad[j])
            dirs += [g, -g]
    return dirs


def _flip_reach(L, allow, p):
    """Smallest multiple lam in (1/8 .. 8) of the allowance field ``allow`` (same
    shape as L) at which one of the candidate directions flips the outcome, or inf."""
    base = _local_decision(L, p)
    dirs = _flip_directions(L, p)
    for lam in (0.125, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 8.0):
        for e in dirs:
            if _local_decision(L + lam * 0.999 * allow * e, p)[0] != base[0]:
                return lam
    return np.inf


@pytest.mark.parametrize("which,rel_scale", [("brain145x174x145", 1.0), ("blobs64", 30.0),
                                             ("brain_crop72x87x72", 30.0)])
def test_every_flagged_voxel_is_within_reach_of_a_flip(detected, monkeypatch, which, rel_scale):
    """Each flagged voxel flips under a perturbation of at most C_TIGHT times the
    allowance (half the tolerance per DoG value).  A flag set padded with voxels
    that no admissible error could move (for example a bound widened by a wrong
    sign or factor) fails here.  On the headline volume this runs at the
    production tolerance; the smaller volumes have few or no near ties at 1e-5,
    so they run with the oracle and this test at 30x the tolerance."""
    res, p = detected
    rel = REL * rel_scale
    vol = brain_like_volume(seed=0) if which == "brain145x174x145" else res[which][0]
    if rel_scale != 1.0:
        monkeypatch.setattr(O, "REL_TOL", rel)
    r = O.detect(vol, p)
    assert r.uncertain, "no flagged voxels: the test checks nothing"
    reach, curv_only = [], []
    for (o, s, z, y, x) in sorted(r.uncertain):
        G, D = r.pyramid.G[o], r.pyramid.D[o]
        L = _local(D, s, z, y, x)
        allow = np.stack([_value_allowance([G[l][z - 1:z + 2, y - 1:y + 2, x - 1:x + 2],
                                            G[l + 1][z - 1:z + 2, y - 1:y + 2, x - 1:x + 2]], rel)[0]
                          for l in (s - 1, s, s + 1)])
        reach.append(_flip_reach(L, allow, p))
        # Which decision has to move: a keypoint flips when any one of its
        # near decisions does; a rejected voxel only when every failing one does.
        mag = max(float(np.max(np.abs(G[l][z - 1:z + 2, y - 1:y + 2, x - 1:x + 2]))) for l in range(s - 1, s + 3))
        tau = rel * mag
        c = L[1, 1, 1, 1]
        exact_near = (np.min(np.abs(np.delete(c - L.reshape(-1), 40))) < tau
                      or abs(abs(c) - p.contrast_thresh) < tau)
        con, ext, curv, _ = _local_tests(L, p)
        keep = con and ext and curv
        curv_only.append(not exact_near if keep else not curv)
    curv_only = np.array(curv_only)
    reach = np.array(reach)
    limit = np.where(curv_only, C_TIGHT_CURV, C_TIGHT)
    far = int(np.sum(reach > limit))
    fin = reach[np.isfinite(reach)]
    q = np.quantile(fin, [0.5, 0.9, 1.0]).tolist() if fin.size else []
    print(f"{which} x{rel_scale}: {len(reach)} flagged ({int(np.sum(curv_only))} by curvature only), "
          f"reach quantiles {q}, beyond the limit: {far}")
    assert far == 0, f"{far} of {len(reach)} flagged voxels are out of reach of a flip; quantiles {q}"
