"""The stored per-scan observation counts that the benchmark turns into
algorithmic bytes (tests/golden/*_counts.json) are the oracle's: recompute
them from the oracle's pair generator on the same seeded inputs (the room
workload in full, the first scans of the differentiation workload) and
check the byte formula on a hand-counted row. CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _pack(ijk):
    i = ijk.astype(np.int64) + (1 << 20)
    return (i[:, 0] << 42) | (i[:, 1] << 21) | i[:, 2]


def _rows(w, n):
    p = oracle.make_params(w.voxel_size, w.trunc, min_range=w.min_range, max_range=w.max_range,
                           body_from_sensor=w.body_from_sensor)
    seen = np.zeros(0, np.int64)
    rows = []
    for s in w.scans[:n]:
        ijk, pt, d = oracle.scan_pairs(p, s["pts"], s["pose"])
        vk = np.unique(_pack(ijk))
        new = int((~np.isin(vk, seen, assume_unique=True)).sum())
        seen = np.union1d(seen, vk)
        rows.append(dict(points=int(s["pts"].shape[0]), valid=int(np.unique(pt).size),
                         pairs=int(d.size), voxels=int(vk.size), new_voxels=new,
                         blocks=int(np.unique(_pack(np.floor_divide(ijk, 8))).size)))
    return rows


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_room_counts_are_the_oracles():
    stored = _load("room_lidar_counts.json")["scans"]
    w = synth.room_lidar(seed=1, n_scans=10)
    assert _rows(w, 10) == stored


def test_adjoint_pair_counts_are_the_oracles():
    stored = _load("adjoint_counts.json")["scans"]
    assert len(stored) == 20
    w = synth.room_lidar(seed=4, n_scans=20, n_beams=64, n_az=2048, K=20, mode="soft")
    got = _rows(w, 2)
    for g, s in zip(got, stored[:2]):
        assert (g["points"], g["valid"], g["pairs"]) == (s["points"], s["valid"], s["pairs"])


def test_indoor_counts_first_frames_are_the_oracles():
    stored = _load("indoor_rgbd_counts.json")
    assert stored["meta"]["frames"] == len(stored["scans"]) == 200
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=8, frames=[0, 1])
    assert _rows(w, 2) == stored["scans"][:2]


@pytest.mark.parametrize("name", ["street_lidar_counts.json", "room_lidar_counts.json",
                                  "indoor_rgbd_counts.json"])
def test_stored_counts_are_consistent(name):
    rows = _load(name)["scans"]
    seen = 0
    for r in rows:
        assert 0 <= r["valid"] <= r["points"]
        assert r["blocks"] <= r["voxels"] <= r["pairs"]
        assert 0 <= r["new_voxels"] <= r["voxels"]
        # a valid point has between 1 and 3 ceil(2 tau / v) + 3 observations
        assert r["valid"] <= r["pairs"]
        seen += r["new_voxels"]
    assert rows[0]["new_voxels"] == rows[0]["voxels"]  # the first scan sees an empty map
    meta = _load(name)["meta"]
    if "total_voxels" in meta:
        assert seen == meta["total_voxels"]


def test_algorithmic_bytes_formula():
    """B = N_all 12 + N_valid 4K + (2 U_old + U_new) R + U_b 16, R = 8 + 4K, on
    a hand-counted row: 10 points, 8 valid, 5 voxels of which 2 new, 1 block,
    K = 2 (R = 16): 120 + 64 + (2 * 3 + 2) * 16 + 16 = 328 bytes."""
    import bench
    counts = {"scans": [dict(points=10, valid=8, pairs=20, voxels=5, new_voxels=2, blocks=1)]}
    assert bench.algorithmic_bytes(counts, 1, K=2) == [328]
    street = _load("street_lidar_counts.json")
    B = bench.algorithmic_bytes(street, 100)
    # 49.1 MB per scan on average; one 16-scan launch of the 100-scan step
    # (7 launches) averages 701.5 MB
    assert abs(sum(B) / 100 / 1e6 - 49.1) < 0.05
    assert abs(sum(B) / 7 / 1e6 - 701.5) < 0.1
