"""Keypoint recall / precision and descriptor agreement of a reduced-precision
run against the FP64 oracle.

A detected keypoint matches an oracle keypoint when both have the same octave
and scale and their grid positions differ by at most one voxel on every axis.
Descriptor agreement is measured on matched pairs whose positions are equal:
the fraction of equal BRIEF bits and of equal RRIEF ranks.
"""
from __future__ import annotations

import numpy as np


def match_keypoints(got, ref, tol: int = 1):
    """Greedy one-to-one matching; returns (pairs, recall, precision)."""
    by_key = {}
    for j, k in enumerate(ref):
        by_key.setdefault((int(k["octave"]), int(k["scale"])), []).append(j)
    used = set()
    pairs = []
    for i, k in enumerate(got):
        cands = by_key.get((int(k["octave"]), int(k["scale"])), [])
        best, bd = None, None
        for j in cands:
            if j in used:
                continue
            r = ref[j]
            d = max(abs(int(k["ix"]) - int(r["ix"])), abs(int(k["iy"]) - int(r["iy"])),
                    abs(int(k["iz"]) - int(r["iz"])))
            if d <= tol and (bd is None or d < bd):
                best, bd = j, d
        if best is not None:
            used.add(best)
            pairs.append((i, best, bd))
    recall = len(pairs) / max(len(ref), 1)
    precision = len(pairs) / max(len(got), 1)
    return pairs, recall, precision


def descriptor_agreement(brief_got, rrief_got, brief_ref, rrief_ref, pairs):
    """Fraction of equal BRIEF bits and RRIEF ranks over exactly co-located pairs."""
    idx = [(i, j) for i, j, d in pairs if d == 0]
    if not idx:
        return 1.0, 1.0
    gi = np.array([i for i, _ in idx])
    rj = np.array([j for _, j in idx])
    bg = (brief_got[gi][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    br = (brief_ref[rj][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    bits = float(np.mean(bg == br))
    ranks = float(np.mean(rrief_got[gi] == rrief_ref[rj]))
    return bits, ranks
