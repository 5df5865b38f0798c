"""Comparison helpers for CUDA-path vs oracle parity (used by the gpu tests).

Tolerances:
* Gaussian and descriptor-blur levels: max |gpu - oracle| <= 1e-5 * max |oracle|
  over the level (float32 arithmetic vs float64).
* DoG levels: max |gpu - oracle| <= 1e-5 * max |G| of that octave (a DoG value is
  a difference of two Gaussian levels, so its error scales with them).
* Keypoint sets: identical except voxels the oracle marks as near ties.
* Descriptors: BRIEF bits identical except |d_k| < 1e-5 * local magnitude; RRIEF
  rank orders identical except pairs with |d_j - d_k| < 1e-5 * local magnitude.
"""
from __future__ import annotations

import numpy as np

REL = 1e-5


def key_set(kps) -> set:
    return {(int(k["octave"]), int(k["scale"]), int(k["iz"]), int(k["iy"]), int(k["ix"])) for k in kps}


def compare_keypoints(got, ref_result):
    """Returns (n_exceptions, report).  Raises AssertionError on an unexplained
    difference."""
    ref = ref_result.keypoints
    g, r = key_set(got), key_set(ref)
    diff = g ^ r
    unexplained = diff - ref_result.uncertain
    assert not unexplained, f"unexplained keypoint differences: {sorted(unexplained)[:10]}"
    # fields of common keypoints
    gi = {(int(k["octave"]), int(k["scale"]), int(k["iz"]), int(k["iy"]), int(k["ix"])): k for k in got}
    n_field_exc = 0
    for k in ref:
        key = (int(k["octave"]), int(k["scale"]), int(k["iz"]), int(k["iy"]), int(k["ix"]))
        if key not in gi:
            continue
        q = gi[key]
        assert q["polarity"] == k["polarity"], key
        if q["sign_sum"] != k["sign_sum"]:
            assert key in ref_result.uncertain, f"sign_sum differs at {key}"
            n_field_exc += 1
        for f in ("x", "y", "z"):
            assert abs(float(q[f]) - float(k[f])) <= 1e-6 * max(1.0, abs(float(k[f]))), (key, f)
        assert abs(float(q["sigma"]) - float(k["sigma"])) <= 1e-6 * float(k["sigma"]), key
    return len(diff) + n_field_exc, {"gpu": len(g), "oracle": len(r), "set_exceptions": len(diff),
                                     "field_exceptions": n_field_exc}


def level_error(gpu: np.ndarray, ref: np.ndarray, scale: float | None = None) -> float:
    s = float(np.max(np.abs(ref))) if scale is None else scale
    return float(np.max(np.abs(gpu.astype(np.float64) - ref))) / max(s, 1e-30)


def compare_descriptors(brief, rrief, dref):
    """brief: (n,) uint64; rrief: (n, 64) uint8; dref: oracle DescribeResult on the
    same keypoints.  Returns the number of exceptions (near-tie comparisons)."""
    n = dref.d.shape[0]
    tol = REL * dref.mag
    bits_ref = ((dref.brief[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(bool)
    bits_got = ((brief[:, None].astype(np.uint64) >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(bool)
    bad = bits_ref != bits_got
    near = np.abs(dref.d) < tol
    assert not np.any(bad & ~near), f"BRIEF bits differ beyond near ties at {np.argwhere(bad & ~near)[:5]}"
    exc = int(np.sum(bad))
    # RRIEF: the order of every pair (j, k) must agree unless d_j ~ d_k
    for i in range(n):
        rg = rrief[i].astype(np.int64)
        rr = dref.rrief[i].astype(np.int64)
        if np.array_equal(rg, rr):
            continue
        d = dref.d[i]
        m = np.maximum(dref.mag[i][:, None], dref.mag[i][None, :])
        order_g = rg[:, None] < rg[None, :]
        order_r = rr[:, None] < rr[None, :]
        wrong = order_g != order_r
        close = np.abs(d[:, None] - d[None, :]) < REL * m
        assert not np.any(wrong & ~close), f"RRIEF order differs beyond near ties for keypoint {i}"
        exc += int(np.sum(wrong)) // 2
        assert sorted(rg.tolist()) == list(range(64))
    return exc
