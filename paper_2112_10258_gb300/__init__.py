"""GB300 (sm_103a) 3D SIFT detector with BRIEF / RRIEF descriptors.

The compute lives in ``libsift3d.so`` (hand-written CUDA, C ABI in
``include/sift3d.h``); this package is its Python binding.  PyTorch is used for
device memory and streams only.
"""
from __future__ import annotations

import numpy as np

from . import capi
from .capi import (DESC_BOTH, DESC_BRIEF, DESC_RRIEF, DTYPE_F32, DTYPE_U8, KEYPOINT_DTYPE, LEVEL_DESC,
                   LEVEL_DOG, LEVEL_GAUSS, STORAGE_BF16, STORAGE_F16, STORAGE_F32, SUBMIT_DEVICE, SUBMIT_NOCOPY,
                   Sift3DError)

__all__ = ["Sift3D", "make_params", "plan", "pattern", "KEYPOINT_DTYPE", "Sift3DError"]


def make_params(**overrides) -> capi.Params:
    p = capi.sift3d_default_params()
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def plan(nx: int, ny: int, nz: int, **overrides) -> dict:
    rc, info = capi.sift3d_plan(make_params(**overrides), nx, ny, nz)
    if rc != capi.OK:
        raise Sift3DError(rc, "sift3d_plan")
    n = info.n_octaves
    L = info.n_levels
    return {
        "n_octaves": n, "n_levels": L,
        "dims": [tuple(info.dims[o]) for o in range(n)],
        "pitch_y": [info.pitch_y[o] for o in range(n)], "pitch_z": [info.pitch_z[o] for o in range(n)],
        "sigma_level": list(info.sigma_level[:L]), "sigma_initial": info.sigma_initial,
        "sigma_increment": list(info.sigma_increment[:L - 1]), "radius_initial": info.radius_initial,
        "radius_increment": list(info.radius_increment[:L - 1]), "radius_desc": info.radius_desc,
        "workspace_bytes": info.workspace_bytes, "algorithmic_bytes": info.algorithmic_bytes,
    }


def pattern(**overrides) -> np.ndarray:
    return capi.sift3d_pattern(make_params(**overrides))


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Sift3D:
    """One library context (pyramid workspace cache, graphs, serving queue)."""

    def __init__(self, **params):
        self.params = make_params(**params)
        rc, self.ctx = capi.sift3d_create(self.params)
        if rc != capi.OK:
            raise Sift3DError(rc, "sift3d_create: invalid parameters")

    def close(self):
        if self.ctx:
            capi.sift3d_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc not in (capi.OK, capi.PENDING):
            raise Sift3DError(rc, f"{what}: {capi.sift3d_last_error(self.ctx)}")
        return rc

    # ---- device API --------------------------------------------------------------
    def detect(self, vol, capacity: int = 16384, out=None, stream=None, sync: bool = True):
        """vol: CUDA tensor (nz, ny, nx) float32 or uint8.  Returns (keypoint byte
        tensor of capacity*48, count or None when sync=False)."""
        import torch
        assert vol.is_cuda and vol.is_contiguous() and vol.dim() == 3
        dtype = DTYPE_U8 if vol.dtype == torch.uint8 else DTYPE_F32
        if dtype == DTYPE_F32 and vol.dtype != torch.float32:
            raise TypeError("vol must be float32 or uint8")
        nz, ny, nx = vol.shape
        if out is None:
            out = torch.empty(max(capacity, 1) * 48, dtype=torch.uint8, device=vol.device)
        rc, n = capi.sift3d_detect(self.ctx, vol.data_ptr(), dtype, nx, ny, nz, _stream_handle(stream),
                                   out.data_ptr(), capacity, want_count=sync)
        if rc == capi.ECAPACITY:
            return out, n
        self._check(rc, "sift3d_detect")
        return out, (n if sync else None)

    def describe(self, kps, n: int = -1, kind: int = DESC_BOTH, stream=None, brief=None, rrief=None,
                 n_alloc: int | None = None):
        import torch
        cap = n_alloc if n_alloc is not None else (n if n >= 0 else kps.numel() // 48)
        dev = kps.device
        if brief is None:
            brief = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        if rrief is None:
            rrief = torch.empty(max(cap, 1) * 64, dtype=torch.uint8, device=dev)
        rc = capi.sift3d_describe(self.ctx, kps.data_ptr(), n, kind, brief.data_ptr(), rrief.data_ptr(),
                                  _stream_handle(stream))
        self._check(rc, "sift3d_describe")
        return brief, rrief

    def describe_siftrank(self, kps, n: int = -1, stream=None, desc=None, rot=None, n_alloc: int | None = None,
                          with_rotation: bool = False):
        """3D SIFT-Rank descriptors (n x 64 uint8 ranks) of keypoints of the last
        detect; with_rotation also returns the n x 9 keypoint frames."""
        import torch
        cap = n_alloc if n_alloc is not None else (n if n >= 0 else kps.numel() // 48)
        dev = kps.device
        if desc is None:
            desc = torch.empty(max(cap, 1) * 64, dtype=torch.uint8, device=dev)
        if with_rotation and rot is None:
            rot = torch.empty(max(cap, 1) * 9, dtype=torch.float32, device=dev)
        rc = capi.sift3d_describe_siftrank(self.ctx, kps.data_ptr(), n, desc.data_ptr(),
                                           rot.data_ptr() if rot is not None else 0, _stream_handle(stream))
        self._check(rc, "sift3d_describe_siftrank")
        return (desc, rot) if with_rotation else desc

    def gaussian_blur(self, vol, sigma: float, out=None, stream=None):
        """Separable 3D Gaussian blur of a dense float32 CUDA tensor (nz, ny, nx)."""
        import torch
        assert vol.is_cuda and vol.dtype == torch.float32 and vol.is_contiguous() and vol.dim() == 3
        nz, ny, nx = vol.shape
        if out is None:
            out = torch.empty_like(vol)
        rc = capi.sift3d_gaussian_blur(self.ctx, vol.data_ptr(), nx, ny, nz, sigma, out.data_ptr(),
                                       _stream_handle(stream))
        self._check(rc, "sift3d_gaussian_blur")
        return out

    def read_level(self, octave: int, kind: int, index: int, dims, stream=None):
        import torch
        nx, ny, nz = dims
        dst = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
        rc = capi.sift3d_read_level(self.ctx, octave, kind, index, dst.data_ptr(), _stream_handle(stream))
        self._check(rc, "sift3d_read_level")
        return dst

    # ---- serving -------------------------------------------------------------------
    def submit(self, host_vol: np.ndarray, flags: int = 0) -> int:
        arr = np.ascontiguousarray(host_vol)
        dtype = DTYPE_U8 if arr.dtype == np.uint8 else DTYPE_F32
        if dtype == DTYPE_F32 and arr.dtype != np.float32:
            raise TypeError("host_vol must be float32 or uint8")
        nz, ny, nx = arr.shape
        rc, t = capi.sift3d_submit(self.ctx, arr.ctypes.data, dtype, nx, ny, nz, flags)
        self._check(rc, "sift3d_submit")
        return t

    def detect_batch(self, vols, capacity: int = 16384, describe: bool = True, stream=None):
        """Detect (and describe) a list of CUDA volumes (float32 or uint8, shapes
        (nz, ny, nx)) in one batched graph launch.  Returns a list of
        (keypoint_buffer, n, brief, rrief) per volume (brief/rrief None when
        describe is False)."""
        import torch
        u8 = vols[0].dtype == torch.uint8
        dims = [(v.shape[2], v.shape[1], v.shape[0]) for v in vols]
        outs = [torch.empty(capacity * 48, dtype=torch.uint8, device="cuda") for _ in vols]
        briefs = [torch.empty(capacity, dtype=torch.int64, device="cuda") for _ in vols] if describe else None
        rriefs = [torch.empty(capacity * 64, dtype=torch.uint8, device="cuda") for _ in vols] if describe else None
        rc, counts = capi.sift3d_detect_batch(self.ctx, [v.data_ptr() for v in vols], dims,
                                              DTYPE_U8 if u8 else DTYPE_F32, _stream_handle(stream),
                                              [o.data_ptr() for o in outs], capacity,
                                              [b.data_ptr() for b in briefs] if describe else None,
                                              [r.data_ptr() for r in rriefs] if describe else None)
        self._check(rc, "sift3d_detect_batch")
        return [(outs[i], counts[i], briefs[i] if describe else None, rriefs[i] if describe else None)
                for i in range(len(vols))]

    def submit_device(self, vol) -> int:
        """Queue a CUDA tensor volume (float32 or uint8, shape (nz, ny, nx)); the
        detect reads it in place, so keep it unchanged until the request ends."""
        import torch
        if not vol.is_cuda or not vol.is_contiguous():
            raise TypeError("vol must be a contiguous CUDA tensor")
        dtype = DTYPE_U8 if vol.dtype == torch.uint8 else DTYPE_F32
        if dtype == DTYPE_F32 and vol.dtype != torch.float32:
            raise TypeError("vol must be float32 or uint8")
        torch.cuda.current_stream().synchronize()   # the volume is complete before submit
        nz, ny, nx = vol.shape
        return self.submit_ptr(vol.data_ptr(), dtype, (nx, ny, nz), flags=SUBMIT_DEVICE)

    def submit_ptr(self, ptr: int, dtype: int, dims, flags: int = 0) -> int:
        nx, ny, nz = dims
        rc, t = capi.sift3d_submit(self.ctx, ptr, dtype, nx, ny, nz, flags)
        self._check(rc, "sift3d_submit")
        return t

    def poll(self, ticket: int, timeout_us: int = 0, copy: bool = True):
        """None while pending; else a dict with numpy copies of the results."""
        rc, r = capi.sift3d_poll(self.ctx, ticket, timeout_us)
        if rc == capi.PENDING:
            return None
        self._check(rc, "sift3d_poll")
        n = r.n_keypoints
        out = {"status": r.status, "n_keypoints": n, "n_needed": r.n_needed,
               "latency_ms": r.latency_ms, "queue_ms": r.queue_ms}
        if copy:
            if n > 0:
                kb = np.ctypeslib.as_array(C_cast(r.keypoints), shape=(n * 48,))
                out["keypoints"] = kb.view(KEYPOINT_DTYPE).copy()
                out["brief"] = np.ctypeslib.as_array(r.brief, shape=(n,)).copy()
                out["rrief"] = np.ctypeslib.as_array(r.rrief, shape=(n * 64,)).reshape(n, 64).copy()
            else:
                out["keypoints"] = np.zeros(0, KEYPOINT_DTYPE)
                out["brief"] = np.zeros(0, np.uint64)
                out["rrief"] = np.zeros((0, 64), np.uint8)
        return out

    def release(self, ticket: int) -> int:
        return capi.sift3d_release(self.ctx, ticket)


def C_cast(ptr):
    import ctypes
    return ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint8))


def match(desc_a, desc_b, kind: int, stream=None, second: bool = True):
    """Nearest neighbour in desc_b of every descriptor of desc_a, on the GPU
    (sift3d_match).  BRIEF: int64/uint64 CUDA tensors of words; RRIEF: uint8
    CUDA tensors of shape (n, 64) (or flat n*64).  Returns int32 CUDA tensors
    (nn, dist, dist2) with dist2 None when second is False."""
    import torch
    if kind == DESC_BRIEF:
        na, nb = desc_a.numel(), desc_b.numel()
    else:
        na, nb = desc_a.numel() // 64, desc_b.numel() // 64
    dev = desc_a.device
    nn = torch.empty(max(na, 1), dtype=torch.int32, device=dev)
    dist = torch.empty(max(na, 1), dtype=torch.int32, device=dev)
    dist2 = torch.empty(max(na, 1), dtype=torch.int32, device=dev) if second else None
    rc = capi.sift3d_match(desc_a.data_ptr(), na, desc_b.data_ptr() if nb > 0 else 0, nb, kind, nn.data_ptr(),
                           dist.data_ptr(), dist2.data_ptr() if second else 0, _stream_handle(stream))
    if rc != capi.OK:
        raise capi.Sift3DError(rc, "sift3d_match")
    return nn[:na], dist[:na], (dist2[:na] if second else None)


def keypoints_to_numpy(buf, n: int) -> np.ndarray:
    """Copy the first n records of a device keypoint byte tensor to a structured array."""
    if n <= 0:
        return np.zeros(0, KEYPOINT_DTYPE)
    return buf[: n * 48].cpu().numpy().view(KEYPOINT_DTYPE).copy()
