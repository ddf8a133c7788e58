"""Write batch_counts.json: per-map, per-scan observation counts of the
batched multi-map workload (8 closed-set street maps and 8 open-set RGB-D
maps, 10 scans each, synth.batch_workload(seed=5)), computed by the oracle's
pair generator only. The benchmark reads them to form the algorithmic bytes
of the batched step; the GPU path does not produce any of them.

Per map: kind (closed / open), width (K classes or l), and per scan: points,
valid, pairs, voxels, new_voxels, blocks (as in make_street_counts.py).

Run: python tests/golden/make_batch_counts.py
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


def map_counts(w):
    p = oracle.make_params(w.voxel_size, w.trunc, min_range=w.min_range, max_range=w.max_range,
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
    return rows


def main(out=os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_counts.json")):
    closed, opened = synth.batch_workload(seed=5, n_scans=10)
    maps = [dict(kind="closed", width=w.num_classes, scans=map_counts(w)) for w in closed]
    maps += [dict(kind="open", width=w.embed_dim, scans=map_counts(w)) for w in opened]
    meta = dict(workload="batch", seed=5, maps=len(maps), scans_per_map=10,
                source="oracle.scan_pairs")
    with open(out, "w") as f:
        json.dump(dict(meta=meta, maps=maps), f, indent=1)
    print(out, meta)


if __name__ == "__main__":
    main()
