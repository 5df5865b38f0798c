"""Reduced-precision storage report (needs a GPU): Gaussian levels stored in
FP32, FP16 and BF16 (arithmetic in FP32, DoG in FP32), on brain-like
145x174x145 volumes of seeds 0..N-1, against the FP64 oracle, beside the recall
and precision of the oracle's FP64 emulation of the same storage arithmetic.

For every storage type it reports keypoint recall and precision (a match is the
same octave and scale with grid positions at most one voxel apart on every
axis), the fraction of equal BRIEF bits and RRIEF ranks over exactly co-located
matches, and the worst relative error of the level G[0][3].

    python -m tests.precision_report --seeds 16 [--out report.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_10258_gb300 as S
    from oracle import sift3d_oracle as O
    from tests.precision import descriptor_agreement, match_keypoints
    from workloads.volumes import brain_like_volume

    p = O.Params()
    storages = (("f32", S.STORAGE_F32), ("f16", S.STORAGE_F16), ("bf16", S.STORAGE_BF16))
    dets = {name: S.Sift3D(storage=code) for name, code in storages}
    acc = {name: {"tp": 0, "n_gpu": 0, "n_ref": 0, "bits": [], "ranks": [], "g_err": 0.0, "recall": [],
                  "precision": [], "emul_tp": 0, "emul_n": 0} for name, _ in storages}
    t0 = time.time()
    for seed in range(args.seeds):
        vol = brain_like_volume(seed=seed)
        ref = O.detect(vol, p)
        dref = O.describe(ref.pyramid, ref.keypoints, p)
        g_ref = ref.pyramid.G[0][3]
        d_vol = torch.from_numpy(vol).cuda()
        for name, _ in storages:
            det = dets[name]
            buf, n = det.detect(d_vol, capacity=16384)
            kps = S.keypoints_to_numpy(buf, n)
            brief, rrief = det.describe(buf, n)
            b = brief[:n].cpu().numpy().view(np.uint64)
            r = rrief[: n * 64].cpu().numpy().reshape(n, 64)
            pairs, recall, precision = match_keypoints(kps, ref.keypoints)
            bits, ranks = descriptor_agreement(b, r, dref.brief, dref.rrief, pairs)
            g = det.read_level(0, S.LEVEL_GAUSS, 3, (145, 174, 145)).cpu().numpy()
            a = acc[name]
            a["tp"] += len(pairs)
            a["n_gpu"] += n
            a["n_ref"] += ref.keypoints.size
            a["bits"].append(bits)
            a["ranks"].append(ranks)
            a["recall"].append(recall)
            a["precision"].append(precision)
            a["g_err"] = max(a["g_err"], float(np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref))))
            if name != "f32":   # the oracle's FP64 emulation of the same storage arithmetic
                e = O.detect_pyramid(O.build_pyramid_stored(vol, p, name), p, keep_pyramid=False)
                ep, _, _ = match_keypoints(e.keypoints, ref.keypoints)
                a["emul_tp"] += len(ep)
                a["emul_n"] += e.keypoints.size
        print(f"seed {seed}: " + "  ".join(
            f"{nm} R={acc[nm]['recall'][-1]:.4f} P={acc[nm]['precision'][-1]:.4f} bits={acc[nm]['bits'][-1]:.4f}"
            for nm, _ in storages), file=sys.stderr, flush=True)
    for d in dets.values():
        d.close()
    report = {"workload": f"brain-like 145x174x145, seeds 0..{args.seeds - 1}", "oracle": "FP64",
              "match": "same octave and scale, |d ix,iy,iz|_inf <= 1", "seconds": round(time.time() - t0, 1)}
    for name, _ in storages:
        a = acc[name]
        report[name] = {"recall": a["tp"] / max(a["n_ref"], 1), "precision": a["tp"] / max(a["n_gpu"], 1),
                        "recall_min_seed": min(a["recall"]), "precision_min_seed": min(a["precision"]),
                        "brief_bit_agreement": float(np.mean(a["bits"])),
                        "rrief_rank_agreement": float(np.mean(a["ranks"])),
                        "keypoints_gpu": a["n_gpu"], "keypoints_oracle": a["n_ref"],
                        "level_g03_max_rel_err": a["g_err"]}
        if name != "f32":
            report[name]["emulation_recall"] = a["emul_tp"] / max(a["n_ref"], 1)
            report[name]["emulation_precision"] = a["emul_tp"] / max(a["emul_n"], 1)
    txt = json.dumps(report)
    print(txt, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
