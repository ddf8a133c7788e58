"""Write indoor_rgbd_counts.json: per-frame observation counts of the 200
frames of the indoor RGB-D workload (640 x 480 pinhole depth, f = 525,
voxel 0.05 m, truncation 0.15 m, seed 3), computed by the oracle's pair
generator only. The benchmark reads them to form the algorithmic bytes of
the open-set integration; the GPU path does not produce any of them.

Per frame: points (all pixels), valid (pixels with >= 1 observation), pairs,
voxels (distinct voxels observed), new_voxels (observed for the first time
in the sequence), blocks (distinct 8^3 blocks observed).

Run: python tests/golden/make_indoor_counts.py
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


def _frame(f):
    """Counts of frame f: (points, valid, pairs, voxel keys, block keys)."""
    # the embedding dimension does not change the geometry (the scene and the
    # rays are drawn before the embeddings), so a small one keeps this fast
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=8, frames=[f])
    s = w.scans[0]
    p = oracle.make_params(w.voxel_size, w.trunc, min_range=w.min_range,
                           max_range=w.max_range, body_from_sensor=w.body_from_sensor)
    ijk, pt, d = oracle.scan_pairs(p, s["pts"], s["pose"])
    return (int(s["pts"].shape[0]), int(np.unique(pt).size), int(d.size), np.unique(pack(ijk)),
            np.unique(pack(np.floor_divide(ijk, 8))), w.voxel_size, w.trunc)


def main(n_frames=200, out=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                        "indoor_rgbd_counts.json")):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_frame, range(n_frames))
    seen = np.zeros(0, np.int64)
    rows = []
    for npts, valid, pairs, vk, bk, vs, tr in res:
        new = int((~np.isin(vk, seen, assume_unique=True)).sum())
        seen = np.union1d(seen, vk)
        rows.append(dict(points=npts, valid=valid, pairs=pairs, voxels=int(vk.size),
                         new_voxels=new, blocks=int(bk.size)))
    meta = dict(workload="indoor-rgbd", seed=3, frames=n_frames, width=640, height=480,
                voxel_size=res[0][5], trunc=res[0][6], total_voxels=int(seen.size),
                source="oracle.scan_pairs")
    with open(out, "w") as f:
        json.dump(dict(meta=meta, scans=rows), f, indent=1)
    print(out, meta)


if __name__ == "__main__":
    main()
