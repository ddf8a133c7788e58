"""Write adjoint_counts.json: per-scan (voxel, point) pair counts of the
differentiation workload (room scene, 20 scans of 64 x 2048 rays, 20 classes,
soft counts, synth.room_lidar(seed=4)), computed by the oracle's pair
generator only. The benchmark reads them to state how much memory a reverse
pass that stored its pair list would hold (16 B per pair: 64-bit voxel key,
32-bit point index, FP32 SDF) beside the measured memory of the recompute
design; the GPU path does not produce any of them.

Run: python tests/golden/make_adjoint_counts.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_12945_gb300 import synth  # noqa: E402


def main(out=os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_counts.json")):
    w = synth.room_lidar(seed=4, n_scans=20, n_beams=64, n_az=2048, K=20, mode="soft")
    p = oracle.make_params(w.voxel_size, w.trunc, min_range=w.min_range, max_range=w.max_range,
                           body_from_sensor=w.body_from_sensor)
    rows = []
    for s in w.scans:
        ijk, pt, d = oracle.scan_pairs(p, s["pts"], s["pose"])
        rows.append(dict(points=int(s["pts"].shape[0]), valid=int(np.unique(pt).size),
                         pairs=int(d.size)))
    meta = dict(workload="adjoint", seed=4, scans=len(rows), source="oracle.scan_pairs")
    with open(out, "w") as f:
        json.dump(dict(meta=meta, scans=rows), f, indent=1)
    print(out, meta, sum(r["pairs"] for r in rows))


if __name__ == "__main__":
    main()
