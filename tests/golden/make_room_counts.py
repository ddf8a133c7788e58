"""Write room_lidar_counts.json: per-scan observation counts of the
10-scan room LiDAR workload (16 beams x 512 azimuths, seed 1), computed
by the oracle's pair generator only. The benchmark reads them to form the
algorithmic bytes of each scan; the GPU path does not produce any of them.

Per scan: points (all inputs), valid (points with >= 1 observation), pairs,
voxels (distinct voxels observed), new_voxels (observed for the first time
in the sequence), blocks (distinct 8^3 blocks observed).

Run: python tests/golden/make_room_counts.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_12945_gb300 import synth  # noqa: E402


def pack(ijk):
    i = ijk.astype(np.int64) + (1 << 20)
    return (i[:, 0] << 42) | (i[:, 1] << 21) | i[:, 2]


def main(n_scans=10, out=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                       "room_lidar_counts.json")):
    w = synth.room_lidar(seed=1, n_scans=n_scans)
    p = oracle.make_params(w.voxel_size, w.trunc, num_classes=w.num_classes,
                           min_range=w.min_range, max_range=w.max_range,
                           body_from_sensor=w.body_from_sensor)
    seen = np.zeros(0, np.int64)
    rows = []
    for s in w.scans:
        ijk, pt, d = oracle.scan_pairs(p, s["pts"], s["pose"])
        vk = np.unique(pack(ijk))
        bk = np.unique(pack(np.floor_divide(ijk, 8)))
        new = int((~np.isin(vk, seen, assume_unique=True)).sum())
        seen = np.union1d(seen, vk)
        rows.append(dict(points=int(s["pts"].shape[0]), valid=int(np.unique(pt).size),
                         pairs=int(d.size), voxels=int(vk.size), new_voxels=new,
                         blocks=int(bk.size)))
    meta = dict(workload="room-lidar", seed=1, scans=n_scans, beams=16, azimuths=512,
                classes=w.num_classes, voxel_size=w.voxel_size, trunc=w.trunc,
                total_voxels=int(seen.size), source="oracle.scan_pairs")
    with open(out, "w") as f:
        json.dump(dict(meta=meta, scans=rows), f, indent=0)
    print(out, meta)


if __name__ == "__main__":
    main()
