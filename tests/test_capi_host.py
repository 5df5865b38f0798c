"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/sift3d.h declares, validates parameters, and its host logic
(octave plan, filter radii, point-pair pattern) agrees with the oracle's
independent implementation."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import sift3d_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sift3d.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_10258_gb300 import capi
    return capi


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sift3d_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for req in ["sift3d_create", "sift3d_destroy", "sift3d_detect", "sift3d_describe", "sift3d_submit",
                "sift3d_poll", "sift3d_last_error"]:
        assert req in names


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    so = lib.LIB_PATH
    handle = ctypes.CDLL(so)
    for n in names:
        assert hasattr(handle, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sift3d_\w+)", out))
    assert set(names) <= exported
    assert set(lib.SIGNATURES) == set(names)


def test_struct_sizes_match_header_layout(lib):
    assert ctypes.sizeof(lib.Keypoint) == 48
    assert lib.KEYPOINT_DTYPE.itemsize == 48
    # offsets the CUDA side writes
    assert lib.Keypoint.dog.offset == 36 and lib.Keypoint.sign_sum.offset == 40
    assert lib.Keypoint.octave.offset == 28 and lib.Keypoint.polarity.offset == 32


def test_default_params(lib):
    p = lib.sift3d_default_params()
    assert math.isclose(p.sigma0, 1.6, rel_tol=1e-6) and math.isclose(p.sigma_in, 0.5)
    assert p.scales_per_octave == 3 and p.sign_sum_min == 80 and p.min_octave_dim == 16
    assert math.isclose(p.desc_blur_sigma, 0.95, rel_tol=1e-6) and p.desc_method == 3
    assert math.isclose(p.contrast_thresh, O.Params().contrast_thresh, rel_tol=1e-6)


@pytest.mark.parametrize("shape", [(145, 174, 145), (64, 64, 64), (33, 17, 40), (256, 256, 192), (15, 80, 80)])
def test_plan_matches_oracle_schedule(lib, shape):
    from paper_2112_10258_gb300 import plan
    nx, ny, nz = shape
    pl = plan(nx, ny, nz)
    op = O.Params()
    oshapes = O.octave_shapes(op, (nz, ny, nx))
    assert pl["n_octaves"] == len(oshapes)
    assert [tuple(d) for d in pl["dims"]] == [(s[2], s[1], s[0]) for s in oshapes]
    np.testing.assert_allclose(pl["sigma_level"], O.level_sigmas(op), rtol=1e-14)
    np.testing.assert_allclose(pl["sigma_increment"], O.increment_sigmas(op), rtol=1e-14)
    assert math.isclose(pl["sigma_initial"], O.initial_sigma(op), rel_tol=1e-14)
    assert pl["radius_initial"] == O.gaussian_radius(O.initial_sigma(op))
    assert pl["radius_increment"] == [O.gaussian_radius(s) for s in O.increment_sigmas(op)]
    assert pl["radius_desc"] == O.gaussian_radius(0.95)
    for o, (x, y, z) in enumerate(pl["dims"]):
        assert pl["pitch_y"][o] % 8 == 0 and pl["pitch_y"][o] >= x
        assert pl["pitch_z"][o] == pl["pitch_y"][o] * y


def test_algorithmic_byte_model(lib):
    from paper_2112_10258_gb300 import plan
    pl = plan(145, 174, 145)
    n = [145 * 174 * 145, 72 * 87 * 72, 36 * 43 * 36, 18 * 21 * 18]
    assert pl["algorithmic_bytes"] == round(84.5 * sum(n) + 4 * n[0])
    assert abs(pl["algorithmic_bytes"] / 1e6 - 367.2) < 0.1
    # 16-bit storage: per octave 11.125 Gaussian-level terms at 2 bytes (base read,
    # 5 writes, 4 re-reads, G_S read, 1/8 next base) and 10 DoG terms at 4 bytes
    # (the DoG stays float32); octave 0 also writes G_0 and reads the float input
    half = plan(145, 174, 145, storage=1)
    assert abs(half["algorithmic_bytes"] - ((11.125 * 2 + 10 * 4) * sum(n) + 4 * n[0])) <= 1
    assert abs(half["algorithmic_bytes"] / 1e6 - 274.3) < 0.1


@pytest.mark.parametrize("seed", [0x5EED5EED, 0, 1234567, 2 ** 63 + 11])
@pytest.mark.parametrize("method", [1, 2, 3, 4, 5])
def test_pattern_matches_oracle_generator(lib, seed, method):
    from paper_2112_10258_gb300 import pattern
    got = pattern(pattern_seed=seed, desc_method=method)
    ref = O.pattern_for(O.Params(desc_method=method, pattern_seed=seed))
    assert got.dtype == np.float32 and got.shape == (64, 2, 3)
    np.testing.assert_array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("field,value", [
    ("sigma0", 0.4), ("scales_per_octave", 0), ("scales_per_octave", 6), ("sign_sum_min", 0),
    ("sign_sum_min", 81), ("border", 0), ("min_octave_dim", 2), ("contrast_thresh", -1.0),
    ("curvature_r", 0.5), ("trunc", 0.0), ("desc_method", 0), ("desc_method", 6), ("storage", 3),
    ("max_inflight", 0),
    ("trunc", 10.0),   # radius ceil(10 * 3.09) > 16
    ("autotune", 2), ("conv_row_tile", 12), ("conv_row_tile", 32), ("conv_z_tile", 4), ("conv_z_tile", 24),
    ("test_wait_timeout", -1), ("refine", 2),
])
def test_invalid_params_rejected(lib, field, value):
    p = lib.sift3d_default_params()
    setattr(p, field, value)
    rc, ctx = lib.sift3d_create(p)
    assert rc == lib.EINVAL and ctx == 0
    rc, _ = lib.sift3d_plan(p, 64, 64, 64)
    assert rc == lib.EINVAL


def test_create_destroy_and_argument_errors_without_device(lib):
    p = lib.sift3d_default_params()
    rc, ctx = lib.sift3d_create(p)
    assert rc == lib.OK and ctx != 0
    # argument checks happen before any device work
    rc, _ = lib.sift3d_detect(ctx, 0, 0, 64, 64, 64, 0, 0, 16)
    assert rc == lib.EINVAL
    assert "NULL" in lib.sift3d_last_error(ctx)
    rc, _ = lib.sift3d_detect(ctx, 1, 7, 64, 64, 64, 0, 1, 16)
    assert rc == lib.EINVAL
    rc, _ = lib.sift3d_detect(ctx, 1, 0, 0, 64, 64, 0, 1, 16)
    assert rc == lib.EINVAL
    assert lib.sift3d_describe(ctx, 1, 5, 3, 1, 1, 0) == lib.EINVAL   # no prior detect
    assert lib.sift3d_read_level(ctx, 0, 0, 0, 1, 0) == lib.EINVAL
    rc, _ = lib.sift3d_poll(ctx, 12345, 0)
    assert rc == lib.ENOTFOUND
    assert lib.sift3d_release(ctx, 12345) == lib.ENOTFOUND
    assert lib.sift3d_device_count(ctx) == 0
    rc, _ = lib.sift3d_plan(p, 64, 64, 4096)
    assert rc == lib.EINVAL
    lib.sift3d_destroy(ctx)
    lib.sift3d_destroy(0)


def test_plan_for_volume_below_min_octave_dim(lib):
    from paper_2112_10258_gb300 import plan
    pl = plan(15, 80, 80)
    assert pl["n_octaves"] == 0 and pl["algorithmic_bytes"] == 0


def test_match_rejects_bad_arguments_without_device(lib):
    from paper_2112_10258_gb300 import capi
    assert capi.sift3d_match(0, 0, 0, 0, 1, 0, 0, 0, 0) == capi.OK          # na == 0: nothing to do
    assert capi.sift3d_match(0, 4, 0, 4, 3, 0, 0, 0, 0) == capi.EINVAL      # kind
    assert capi.sift3d_match(0, -1, 0, 4, 1, 0, 0, 0, 0) == capi.EINVAL     # negative count
    assert capi.sift3d_match(0, 4, 0, 4, 1, 0, 0, 0, 0) == capi.EINVAL      # NULL pointers
    assert capi.sift3d_match(8, 4, 8, 4, 2, 16, 16, 0, 0) == capi.EINVAL    # RRIEF rows not 16-byte aligned


def test_allocation_failure_hook_arguments(lib):
    """The test hook takes n >= 0 (0 cancels) and needs no device."""
    from paper_2112_10258_gb300 import capi
    assert capi.sift3d_test_fail_allocation(-1) == capi.EINVAL
    assert capi.sift3d_test_fail_allocation(5) == capi.OK
    assert capi.sift3d_test_fail_allocation(0) == capi.OK
