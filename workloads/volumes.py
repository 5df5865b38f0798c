"""Seeded synthetic input volumes shared by the CUDA path's tests/bench and the oracle.

This module only *makes inputs*; it holds none of the detector's arithmetic (no
scale-space, DoG, extremum or descriptor code).  Arrays are returned in the memory
layout the library uses: numpy shape (nz, ny, nx), C order, x fastest.

The paper's workload is OASIS-1 T1 brain MRI at 145x174x145 voxels with ~2900
keypoints per volume (Sec. 2.3, Table 2).  That dataset is not available here, so
these generators stand in for it:

* ``blob_volume``   - isotropic Gaussian blobs plus white noise (64^3 detect case).
* ``brain_like_volume`` - nested ellipsoid shells (0.2/0.5/0.8) warped by a smooth
  random displacement field, small blobs at a minimum spacing (6500 on
  145x174x145), and Rician-like magnitude noise.
* ``batch_shapes`` / ``poisson_arrivals`` - uneven batch sizes and a request stream.

The smoothing of the displacement field uses an FFT-domain Gaussian transfer
function, unrelated to the spatial FIR filters the detector uses.
"""
from __future__ import annotations

import numpy as np

BRAIN_SHAPE = (145, 174, 145)  # (nx, ny, nz), Sec. 2.3 / abstract


def blob_volume(seed: int = 0, shape=(64, 64, 64), n_blobs: int = 40,
                sigma_range=(2.0, 6.0), amp_range=(0.5, 1.0), noise_std: float = 0.01,
                dtype=np.float32) -> np.ndarray:
    """Sum of ``n_blobs`` isotropic Gaussians (sigma ~ U[sigma_range], amplitude
    +-U[amp_range], centres uniform in the volume) plus N(0, noise_std^2) noise."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    vol = np.zeros((nz, ny, nx), np.float64)
    centres = rng.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1], size=(n_blobs, 3))
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_blobs)
    amps = rng.uniform(amp_range[0], amp_range[1], size=n_blobs)
    amps *= np.where(rng.random(n_blobs) < 0.5, -1.0, 1.0)
    _splat_blobs(vol, centres, sigmas, amps)
    vol += rng.normal(0.0, noise_std, size=vol.shape)
    return vol.astype(dtype)


def _splat_blobs(vol: np.ndarray, centres, sigmas, amps, extent: float = 4.0) -> None:
    """Add A*exp(-r^2/(2 s^2)) for each blob inside a +-extent*s box."""
    nz, ny, nx = vol.shape
    for (cx, cy, cz), s, a in zip(centres, sigmas, amps):
        r = int(np.ceil(extent * s))
        x0, x1 = max(0, int(np.floor(cx)) - r), min(nx, int(np.floor(cx)) + r + 2)
        y0, y1 = max(0, int(np.floor(cy)) - r), min(ny, int(np.floor(cy)) + r + 2)
        z0, z1 = max(0, int(np.floor(cz)) - r), min(nz, int(np.floor(cz)) + r + 2)
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        gx = np.exp(-((np.arange(x0, x1) - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((np.arange(y0, y1) - cy) ** 2) / (2 * s * s))
        gz = np.exp(-((np.arange(z0, z1) - cz) ** 2) / (2 * s * s))
        vol[z0:z1, y0:y1, x0:x1] += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]


def _smooth_noise_fft(rng, shape_zyx, sigma: float) -> np.ndarray:
    """White noise low-passed by the Gaussian transfer function exp(-2 pi^2 s^2 |f|^2)."""
    nz, ny, nx = shape_zyx
    n = rng.standard_normal(shape_zyx)
    f = np.fft.rfftn(n)
    fz = np.fft.fftfreq(nz)[:, None, None]
    fy = np.fft.fftfreq(ny)[None, :, None]
    fx = np.fft.rfftfreq(nx)[None, None, :]
    f *= np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * (fx ** 2 + fy ** 2 + fz ** 2))
    return np.fft.irfftn(f, s=shape_zyx, axes=(0, 1, 2))


BLOB_DENSITY = 6500 / (145 * 174 * 145)   # blobs per voxel of the brain-like family


def _spaced_centres(rng, n: int, shape_xyz, min_dist: float) -> np.ndarray:
    """Up to ``n`` centres uniform in the box, each at least ``min_dist`` from
    every earlier one (dart throwing over a grid of cells of side min_dist/sqrt(3),
    which holds at most one centre each)."""
    nx, ny, nz = shape_xyz
    if n <= 0:
        return np.zeros((0, 3))
    if min_dist <= 0:
        return rng.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1], size=(n, 3))
    cell = min_dist / np.sqrt(3.0)
    grid = {}
    out = []
    reach = int(np.ceil(min_dist / cell))
    d2 = min_dist * min_dist
    tries = 0
    while len(out) < n and tries < 20 * n:
        batch = rng.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1], size=(1024, 3))
        for c in batch:
            tries += 1
            key = (int(c[0] // cell), int(c[1] // cell), int(c[2] // cell))
            ok = True
            for dx in range(-reach, reach + 1):
                for dy in range(-reach, reach + 1):
                    for dz in range(-reach, reach + 1):
                        q = grid.get((key[0] + dx, key[1] + dy, key[2] + dz))
                        if q is not None and (q[0] - c[0]) ** 2 + (q[1] - c[1]) ** 2 + (q[2] - c[2]) ** 2 < d2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                grid[key] = c
                out.append(c)
                if len(out) == n:
                    break
    return np.array(out).reshape(-1, 3)


def brain_like_volume(seed: int = 0, shape=BRAIN_SHAPE, warp_sigma: float = 8.0,
                      warp_rms: float = 3.0, semi_axes=(0.45, 0.35, 0.22),
                      intensities=(0.2, 0.5, 0.8), n_blobs: int | None = None,
                      blob_sigma=(2.2, 3.5), blob_amp=(0.2, 0.6), blob_min_dist: float = 6.8,
                      noise_std: float = 0.02, dtype=np.float32) -> np.ndarray:
    """Brain-MRI-shaped stand-in for an OASIS-1 T1 volume.

    Nested ellipsoids with semi-axes ``semi_axes`` x dims (outer to inner) hold
    intensities 0.2/0.5/0.8; the sampling coordinates are displaced by a smooth
    random field (white noise smoothed at ``warp_sigma`` voxels, scaled so the
    vector field has ``warp_rms`` voxels RMS); ``n_blobs`` Gaussian blobs (by
    default 6500 per 145x174x145 voxels, the same density for other shapes)
    with sigma ~ U[blob_sigma], amplitude +-U[blob_amp] and centres uniform but
    at least ``blob_min_dist`` voxels apart are added; finally Rician-like
    magnitude noise |I + n1 + i n2|, n ~ N(0, noise_std^2).  The defaults give
    about 2900 keypoints on 145x174x145 under the default detector parameters,
    the paper's per-volume average.
    """
    nx, ny, nz = shape
    if n_blobs is None:
        n_blobs = int(round(BLOB_DENSITY * nx * ny * nz))
    rng = np.random.default_rng(seed)
    zyx = (nz, ny, nx)
    d = np.stack([_smooth_noise_fft(rng, zyx, warp_sigma) for _ in range(3)])
    d *= warp_rms / np.sqrt(np.mean(np.sum(d * d, axis=0)))
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    px = x + d[0] - (nx - 1) / 2.0
    py = y + d[1] - (ny - 1) / 2.0
    pz = z + d[2] - (nz - 1) / 2.0
    del d, x, y, z
    vol = np.zeros(zyx, np.float64)
    for frac, inten in zip(semi_axes, intensities):
        ax, ay, az = frac * nx, frac * ny, frac * nz
        inside = (px / ax) ** 2 + (py / ay) ** 2 + (pz / az) ** 2 <= 1.0
        vol[inside] = inten
    del px, py, pz
    centres = _spaced_centres(rng, n_blobs, (nx, ny, nz), blob_min_dist)
    m = len(centres)
    sigmas = rng.uniform(blob_sigma[0], blob_sigma[1], size=m)
    amps = rng.uniform(blob_amp[0], blob_amp[1], size=m)
    amps *= np.where(rng.random(m) < 0.5, -1.0, 1.0)
    _splat_blobs(vol, centres, sigmas, amps)
    n1 = rng.normal(0.0, noise_std, size=zyx)
    n2 = rng.normal(0.0, noise_std, size=zyx)
    vol = np.sqrt((vol + n1) ** 2 + n2 ** 2)
    return vol.astype(dtype)


def to_uint8(vol: np.ndarray) -> np.ndarray:
    """Quantise a non-negative volume to uint8 codes (scanner-style 8-bit input)."""
    peak = float(np.max(vol)) if vol.size else 1.0
    peak = peak if peak > 0 else 1.0
    return np.clip(np.rint(vol / peak * 255.0), 0, 255).astype(np.uint8)


def batch_shapes(n: int = 256, lo: int = 96, hi: int = 256, seed: int = 0):
    """Per-axis sizes uniform on {lo..hi} for ``n`` volumes, as (nx, ny, nz) tuples."""
    rng = np.random.default_rng(seed)
    s = rng.integers(lo, hi + 1, size=(n, 3))
    return [tuple(int(v) for v in row) for row in s]


SERVING_SHAPES = ((64, 64, 64), BRAIN_SHAPE, (256, 256, 192))


def poisson_arrivals(n: int, rate_per_s: float = 200.0, seed: int = 0,
                     shapes=SERVING_SHAPES):
    """A request stream: exponential inter-arrival gaps (Poisson process at
    ``rate_per_s``) and shapes drawn with equal probability from ``shapes``.
    Returns a list of (arrival_time_s, (nx, ny, nz))."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    t = np.cumsum(gaps) - gaps[0]
    idx = rng.integers(0, len(shapes), size=n)
    return [(float(t[i]), tuple(shapes[idx[i]])) for i in range(n)]


def batch_volumes(n: int = 256, lo: int = 96, hi: int = 256, n_bases: int = 4, seed: int = 0):
    """``n`` volumes of the brain-like family with per-axis sizes on {lo..hi}.

    Generating hundreds of brain-like volumes one by one takes minutes of host
    time, so ``n_bases`` hi^3 volumes are generated (seeds seed .. seed+n_bases-1)
    and volume i is a box of shape ``batch_shapes(n, lo, hi, seed)[i]`` cut from
    base i % n_bases at an offset drawn uniformly from the positions where it
    fits.  Yields (i, (nx, ny, nz), contiguous float32 array) lazily, so callers
    can upload each volume and drop the host copy.
    """
    shapes = batch_shapes(n, lo, hi, seed)
    bases = [brain_like_volume(seed=seed + b, shape=(hi, hi, hi)) for b in range(n_bases)]
    rng = np.random.default_rng(seed + 1_000_003)
    for i, (nx, ny, nz) in enumerate(shapes):
        ox = int(rng.integers(0, hi - nx + 1))
        oy = int(rng.integers(0, hi - ny + 1))
        oz = int(rng.integers(0, hi - nz + 1))
        yield i, (nx, ny, nz), np.ascontiguousarray(bases[i % n_bases][oz:oz + nz, oy:oy + ny, ox:ox + nx])
