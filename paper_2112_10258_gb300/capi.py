"""ctypes binding of include/sift3d.h.

Argument marshalling only: every step of the detector runs in the CUDA library.
The functions keep the C names (``sift3d_create``, ``sift3d_detect`` ...) and take
plain Python ints for device pointers and streams.  Importing this module loads
``_build/libsift3d.so`` and raises if it is missing - there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsift3d.so")

OK, PENDING = 0, 1
EINVAL, ENOMEM, ECAPACITY, ETIMEDOUT, ECUDA, ENOTFOUND, EBUDGET = -1, -2, -3, -4, -5, -6, -7
DTYPE_F32, DTYPE_U8 = 0, 1
STORAGE_F32, STORAGE_F16, STORAGE_BF16 = 0, 1, 2
DESC_BRIEF, DESC_RRIEF, DESC_BOTH = 1, 2, 3
LEVEL_GAUSS, LEVEL_DOG, LEVEL_DESC = 0, 1, 2
SUBMIT_NOCOPY, SUBMIT_DEVICE = 1, 2
MAX_OCTAVES, MAX_SCALES, N_PAIRS = 16, 5, 64

STATUS_NAMES = {OK: "OK", PENDING: "PENDING", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECAPACITY: "ECAPACITY",
                ETIMEDOUT: "ETIMEDOUT", ECUDA: "ECUDA", ENOTFOUND: "ENOTFOUND", EBUDGET: "EBUDGET"}


class Params(C.Structure):
    _fields_ = [
        ("sigma0", C.c_double), ("sigma_in", C.c_double), ("scales_per_octave", C.c_int32),
        ("min_octave_dim", C.c_int32), ("max_octaves", C.c_int32), ("sign_sum_min", C.c_int32),
        ("border", C.c_int32), ("profile", C.c_int32), ("contrast_thresh", C.c_double),
        ("curvature_r", C.c_double), ("trunc", C.c_double), ("desc_blur_sigma", C.c_double),
        ("desc_method", C.c_int32),
        ("pattern_seed", C.c_uint64), ("storage", C.c_int32), ("use_graphs", C.c_int32),
        ("hbm_budget_bytes", C.c_uint64), ("max_keypoints", C.c_int32), ("max_inflight", C.c_int32),
        ("refine", C.c_int32), ("test_wait_timeout", C.c_int32), ("autotune", C.c_int32),
        ("conv_row_tile", C.c_int32), ("conv_z_tile", C.c_int32),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("n_octaves", C.c_int32), ("n_levels", C.c_int32), ("dims", (C.c_int32 * 3) * MAX_OCTAVES),
        ("pitch_y", C.c_int64 * MAX_OCTAVES), ("pitch_z", C.c_int64 * MAX_OCTAVES),
        ("sigma_level", C.c_double * (MAX_SCALES + 3)), ("sigma_initial", C.c_double),
        ("sigma_increment", C.c_double * (MAX_SCALES + 3)), ("radius_initial", C.c_int32),
        ("radius_increment", C.c_int32 * (MAX_SCALES + 3)), ("radius_desc", C.c_int32),
        ("workspace_bytes", C.c_uint64), ("algorithmic_bytes", C.c_uint64),
    ]


class Keypoint(C.Structure):
    _fields_ = [
        ("x", C.c_float), ("y", C.c_float), ("z", C.c_float), ("sigma", C.c_float),
        ("ix", C.c_int32), ("iy", C.c_int32), ("iz", C.c_int32), ("octave", C.c_int16),
        ("scale", C.c_int16), ("polarity", C.c_int8), ("refined", C.c_int8), ("reserved0", C.c_int8 * 2),
        ("dog", C.c_float),
        ("sign_sum", C.c_int32), ("reserved1", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("n_keypoints", C.c_int32), ("n_needed", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("keypoints", C.POINTER(Keypoint)), ("brief", C.POINTER(C.c_uint64)), ("rrief", C.POINTER(C.c_uint8)),
        ("latency_ms", C.c_double), ("queue_ms", C.c_double),
    ]


KEYPOINT_DTYPE = np.dtype([
    ("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("sigma", "<f4"), ("ix", "<i4"), ("iy", "<i4"),
    ("iz", "<i4"), ("octave", "<i2"), ("scale", "<i2"), ("polarity", "i1"), ("refined", "i1"), ("reserved0", "i1", (2,)),
    ("dog", "<f4"), ("sign_sum", "<i4"), ("reserved1", "<i4"),
])
assert KEYPOINT_DTYPE.itemsize == C.sizeof(Keypoint) == 48

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "sift3d_default_params": (C.c_int, [C.POINTER(Params)]),
    "sift3d_plan": (C.c_int, [C.POINTER(Params), C.c_int, C.c_int, C.c_int, C.POINTER(PlanInfo)]),
    "sift3d_pattern": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_float)]),
    "sift3d_create": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "sift3d_destroy": (None, [C.c_void_p]),
    "sift3d_last_error": (C.c_char_p, [C.c_void_p]),
    "sift3d_detect": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "sift3d_device_count": (C.c_void_p, [C.c_void_p]),
    "sift3d_describe": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "sift3d_read_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "sift3d_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                C.POINTER(C.c_uint64)]),
    "sift3d_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(Result)]),
    "sift3d_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sift3d_gaussian_blur": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_void_p, C.c_void_p]),
    "sift3d_gaussian_blur_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                               C.c_void_p, C.c_void_p]),
    "sift3d_stage_times": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_char_p),
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_int)]),
    "sift3d_stage_timeline": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                        C.POINTER(C.c_int)]),
    "sift3d_match": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p]),
    "sift3d_describe_siftrank": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sift3d_test_fail_allocation": (C.c_int, [C.c_int]),
    "sift3d_detect_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.c_int,
                                      C.c_void_p, C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libsift3d.so not built ({path}); run __graft_entry__.build() or "
                          "python paper_2112_10258_gb300/build.py")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class Sift3DError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


# ---- same-named wrappers (marshalling only) ----------------------------------------

def sift3d_default_params() -> Params:
    p = Params()
    _lib.sift3d_default_params(C.byref(p))
    return p


def sift3d_plan(params: Params, nx: int, ny: int, nz: int) -> tuple[int, PlanInfo]:
    info = PlanInfo()
    return _lib.sift3d_plan(C.byref(params), nx, ny, nz, C.byref(info)), info


def sift3d_pattern(params: Params) -> np.ndarray:
    buf = (C.c_float * (N_PAIRS * 6))()
    rc = _lib.sift3d_pattern(C.byref(params), buf)
    if rc != OK:
        raise Sift3DError(rc, "sift3d_pattern")
    return np.frombuffer(buf, np.float32).reshape(N_PAIRS, 2, 3).copy()


def sift3d_create(params: Params) -> tuple[int, int]:
    h = C.c_void_p()
    rc = _lib.sift3d_create(C.byref(params), C.byref(h))
    return rc, (h.value or 0)


def sift3d_destroy(ctx: int) -> None:
    _lib.sift3d_destroy(C.c_void_p(ctx))


def sift3d_last_error(ctx: int) -> str:
    s = _lib.sift3d_last_error(C.c_void_p(ctx))
    return s.decode() if s else ""


def sift3d_detect(ctx, dev_vol, dtype, nx, ny, nz, stream, dev_out, capacity, want_count=True):
    n = C.c_int(0)
    rc = _lib.sift3d_detect(C.c_void_p(ctx), C.c_void_p(dev_vol), dtype, nx, ny, nz, C.c_void_p(stream),
                            C.c_void_p(dev_out), capacity, C.byref(n) if want_count else None)
    return rc, n.value


def sift3d_device_count(ctx) -> int:
    return _lib.sift3d_device_count(C.c_void_p(ctx)) or 0


def sift3d_describe(ctx, dev_kps, n, kind, dev_brief, dev_rrief, stream) -> int:
    return _lib.sift3d_describe(C.c_void_p(ctx), C.c_void_p(dev_kps), n, kind, C.c_void_p(dev_brief),
                                C.c_void_p(dev_rrief), C.c_void_p(stream))


def sift3d_gaussian_blur(ctx, dev_in, nx, ny, nz, sigma, dev_out, stream) -> int:
    return _lib.sift3d_gaussian_blur(C.c_void_p(ctx), C.c_void_p(dev_in), nx, ny, nz, float(sigma),
                                     C.c_void_p(dev_out), C.c_void_p(stream))


def sift3d_gaussian_blur_noalloc(dev_in, nx, ny, nz, sigma, trunc, dev_out, stream) -> int:
    return _lib.sift3d_gaussian_blur_noalloc(C.c_void_p(dev_in), nx, ny, nz, float(sigma), float(trunc),
                                             C.c_void_p(dev_out), C.c_void_p(stream))


def sift3d_read_level(ctx, octave, kind, index, dev_dst, stream) -> int:
    return _lib.sift3d_read_level(C.c_void_p(ctx), octave, kind, index, C.c_void_p(dev_dst), C.c_void_p(stream))


def sift3d_detect_batch(ctx, vol_ptrs, dims, dtype, stream, out_ptrs, capacity, brief_ptrs=None, rrief_ptrs=None,
                        want_counts=True):
    """Batched detect (+ describe when brief_ptrs/rrief_ptrs are given): device
    pointers per volume, dims as [(nx, ny, nz), ...]; returns (rc, counts)."""
    n = len(vol_ptrs)
    P = C.c_void_p * n
    d = (C.c_int * (3 * n))(*[v for xyz in dims for v in xyz])
    counts = (C.c_int * n)()
    bp = P(*brief_ptrs) if brief_ptrs is not None else None
    rp = P(*rrief_ptrs) if rrief_ptrs is not None else None
    rc = _lib.sift3d_detect_batch(C.c_void_p(ctx), n, P(*vol_ptrs), d, dtype, C.c_void_p(stream), P(*out_ptrs),
                                  capacity, bp, rp, counts if want_counts else None)
    return rc, list(counts)


def sift3d_test_fail_allocation(n: int) -> int:
    return _lib.sift3d_test_fail_allocation(n)


def sift3d_submit(ctx, host_vol_ptr, dtype, nx, ny, nz, flags=0) -> tuple[int, int]:
    t = C.c_uint64(0)
    rc = _lib.sift3d_submit(C.c_void_p(ctx), C.c_void_p(host_vol_ptr), dtype, nx, ny, nz, flags, C.byref(t))
    return rc, t.value


def sift3d_poll(ctx, ticket, timeout_us) -> tuple[int, Result]:
    r = Result()
    rc = _lib.sift3d_poll(C.c_void_p(ctx), ticket, timeout_us, C.byref(r))
    return rc, r


def sift3d_release(ctx, ticket) -> int:
    return _lib.sift3d_release(C.c_void_p(ctx), ticket)


def sift3d_stage_times(ctx, max_n: int = 512):
    """Returns (rc, [(label, ms, algorithmic_bytes), ...]) for the last detect."""
    ms = (C.c_float * max_n)()
    names = (C.c_char_p * max_n)()
    ab = (C.c_uint64 * max_n)()
    n = C.c_int(0)
    rc = _lib.sift3d_stage_times(C.c_void_p(ctx), max_n, ms, names, ab, C.byref(n))
    if rc != OK:
        return rc, []
    k = min(n.value, max_n)
    return rc, [(names[i].decode(), float(ms[i]), int(ab[i])) for i in range(k)]


def sift3d_stage_timeline(ctx, max_n: int = 512):
    """Returns (rc, [(begin_ms, end_ms), ...]) for the last profiled detect,
    relative to the first kernel's begin; same order as sift3d_stage_times."""
    b = (C.c_float * max_n)()
    e = (C.c_float * max_n)()
    n = C.c_int(0)
    rc = _lib.sift3d_stage_timeline(C.c_void_p(ctx), max_n, b, e, C.byref(n))
    if rc != OK:
        return rc, []
    k = min(n.value, max_n)
    return rc, [(float(b[i]), float(e[i])) for i in range(k)]


def sift3d_match(dev_a: int, na: int, dev_b: int, nb: int, kind: int, dev_nn: int, dev_dist: int, dev_dist2: int,
                 stream: int) -> int:
    """Nearest-neighbour matching; pointers are device addresses (0 = NULL)."""
    return _lib.sift3d_match(C.c_void_p(dev_a), na, C.c_void_p(dev_b), nb, kind, C.c_void_p(dev_nn),
                             C.c_void_p(dev_dist), C.c_void_p(dev_dist2), C.c_void_p(stream))


def sift3d_describe_siftrank(ctx, dev_kps: int, n: int, dev_desc: int, dev_rot: int, stream: int) -> int:
    return _lib.sift3d_describe_siftrank(C.c_void_p(ctx), C.c_void_p(dev_kps), n, C.c_void_p(dev_desc),
                                         C.c_void_p(dev_rot), C.c_void_p(stream))
