"""Closed-set parity of the CUDA path against the oracle (element by element,
bit-exact voxel sets, weights and one-hot counts; FP32 D, soft counts and
posteriors within 1e-5 relative / 1e-6 absolute)."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import RTOL, ATOL, assert_close, compare_closed, gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


@pytest.mark.parametrize("agg", ["sort", "hash", "direct"])
def test_room_lidar_onehot(agg):
    w = synth.room_lidar(n_scans=10)
    g = to_np(gpu_map(w, aggregation=agg).extract())
    o = oracle_map(w).extract()
    compare_closed(g, o, "onehot")
    assert np.array_equal(g["sem"].sum(1), g["W"])


def test_room_posterior_and_alpha0():
    w = synth.room_lidar(n_scans=3, n_beams=16, n_az=256)
    for a0 in (0.0, 1.0):
        gm = gpu_map(w, alpha0=a0)
        g = to_np(gm.extract(posterior=True))
        o = oracle_map(w, alpha0=a0).extract(posterior=True)
        assert np.array_equal(g["ijk"], o["ijk"])
        assert_close(g["sem"], o["sem"], RTOL, ATOL, "posterior")
        assert_close(g["sem"].sum(1), np.ones(len(g["W"])), 1e-5, 1e-6, "posterior sum")


@pytest.mark.parametrize("agg,tile", [("sort", 0), ("hash", 64), ("hash", 128), ("hash", 256),
                                      ("direct", 0)])
def test_street_lidar_reduced(agg, tile):
    w = synth.street_lidar(n_scans=4, n_beams=64, n_az=512)
    g = to_np(gpu_map(w, aggregation=agg, tile_points=tile).extract())
    o = oracle_map(w).extract()
    compare_closed(g, o, "onehot")


@pytest.mark.parametrize("agg", ["sort", "direct"])
def test_soft_counts(agg):
    w = synth.room_lidar(n_scans=4, n_beams=16, n_az=256, K=20, mode="soft")
    g = to_np(gpu_map(w, mode="soft", aggregation=agg).extract())
    o = oracle_map(w, mode="soft").extract()
    compare_closed(g, o, "soft")


@pytest.mark.parametrize("agg", ["sort", "hash", "direct"])
def test_ragged_empty_and_invalid(agg):
    """n = 0, single points, a ragged tail, NaN / out-of-range points."""
    w = synth.room_lidar(n_scans=2, n_beams=16, n_az=64)
    s0 = w.scans[0]
    pts = s0["pts"].copy()
    pts[5] = np.nan
    pts[7] = [1e9, 0, 0]
    pts[9] = [0.01, 0, 0]
    scans = [dict(pts=pts[:0], pose=s0["pose"], sem=s0["sem"][:0]),
             dict(pts=pts[:1], pose=s0["pose"], sem=s0["sem"][:1]),
             dict(pts=pts[:777], pose=s0["pose"], sem=s0["sem"][:777]),
             w.scans[1]]
    w.scans = scans
    g = to_np(gpu_map(w, aggregation=agg).extract())
    o = oracle_map(w).extract()
    compare_closed(g, o, "onehot")


def test_empty_map_extract():
    w = synth.room_lidar(n_scans=1, n_beams=4, n_az=8)
    w.scans = [dict(pts=np.zeros((0, 3), np.float32), pose=w.scans[0]["pose"],
                    sem=np.zeros((0, 10), np.float32))]
    m = gpu_map(w)
    ext = m.extract()
    assert ext["W"].shape[0] == 0


@pytest.mark.parametrize("agg", ["sort", "hash", "direct"])
def test_block_capacity_fault_is_reported(agg):
    """Too few blocks: the sticky status reports SLIM_ERR_CAPACITY; nothing hangs."""
    from paper_2512_12945_gb300 import slim
    w = synth.room_lidar(n_scans=1)
    m = slim.Map(voxel_size=0.1, trunc=0.3, num_classes=10, min_range=0.1, max_range=100.0,
                 block_capacity=16, max_points=w.scans[0]["pts"].shape[0], aggregation=agg)
    s = w.scans[0]
    m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
    with pytest.raises(slim.SlimError) as e:
        m.sync()
    assert e.value.status == 3
    assert m.stats()["status"] == 3
    m.reset()
    m.sync()  # reset clears the status


def test_host_entry_point_matches_device_and_oracle():
    """slim_integrate_host from pinned host buffers, six calls in a row (the
    two staging buffers are each reused while the other call's copies run):
    the same map as the device entry point and the oracle."""
    w = synth.room_lidar(n_scans=6, n_beams=16, n_az=256)
    from paper_2512_12945_gb300 import slim
    a = gpu_map(w)
    b = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=10, min_range=w.min_range,
                 max_range=w.max_range, max_points=w.scans[0]["pts"].shape[0])
    host = [(torch.from_numpy(s["pts"]).pin_memory(), torch.from_numpy(s["sem"]).pin_memory())
            for s in w.scans]
    for (p, q), s in zip(host, w.scans):
        b.integrate_host(p, s["pose"], q)
    b.sync()
    ga, gb = to_np(a.extract()), to_np(b.extract())
    assert np.array_equal(ga["ijk"], gb["ijk"]) and np.array_equal(ga["W"], gb["W"])
    assert_close(ga["D"], gb["D"], RTOL, ATOL, "D")
    compare_closed(gb, oracle_map(w).extract(), "onehot")


@pytest.mark.parametrize("agg", ["sort", "hash"])
def test_full_size_street_scans_parity(agg):
    """Full launch configuration: 64 x 2048 scans (131,072 points per call)."""
    w = synth.street_lidar(n_scans=2)
    g = to_np(gpu_map(w, aggregation=agg).extract())
    o = oracle_map(w).extract()
    compare_closed(g, o, "onehot")


def test_wide_band_and_hash_collisions():
    """tau = 4 voxels (the widest band: 30-step cap, 128-point tiles) and a
    tiny hash table (long probe runs) still match the oracle."""
    w = synth.room_lidar(n_scans=3, n_beams=16, n_az=256)
    w.trunc = 0.4
    for agg, tile in (("sort", 0), ("hash", 64), ("hash", 256)):
        g = to_np(gpu_map(w, aggregation=agg, tile_points=tile, hash_capacity=4096,
                          block_capacity=3000).extract())
        o = oracle_map(w).extract()
        compare_closed(g, o, "onehot")


def test_full_size_100_scans_invariants():
    """The benchmark workload (100 full scans): every voxel has sum c = W, D in
    [-tau, tau], and the total weight equals the oracle's pair count."""
    w = synth.street_lidar(n_scans=100)
    g = to_np(gpu_map(w, block_capacity=400000, hash_capacity=1 << 21).extract())
    assert np.array_equal(g["sem"].sum(1), g["W"])
    assert (np.abs(g["D"]) <= np.float32(0.3) + 1e-6).all()
    p = oracle.make_params(w.voxel_size, w.trunc, num_classes=20, min_range=w.min_range,
                           max_range=w.max_range, body_from_sensor=w.body_from_sensor)
    total = 0
    for s in w.scans[::10]:
        total += len(oracle.scan_pairs(p, s["pts"], s["pose"])[2])
    sub = gpu_map(w, scans=w.scans[::10], block_capacity=400000, hash_capacity=1 << 21)
    assert float(to_np(sub.extract())["W"].sum()) == total


def test_autotune_picks_a_tile_and_resets():
    from paper_2512_12945_gb300 import slim
    w = synth.street_lidar(n_scans=2)
    s = w.scans[0]
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=20, min_range=w.min_range,
                 max_range=w.max_range, body_from_sensor=w.body_from_sensor, max_points=131072)
    pts, sem = torch.from_numpy(s["pts"]).cuda(), torch.from_numpy(s["sem"]).cuda()
    best = m.autotune(pts, s["pose"], sem)
    assert best in (0, 64, 128, 256)  # 0: direct reductions
    assert m.stats()["blocks"] == 0
    for sc in w.scans:
        m.integrate(torch.from_numpy(sc["pts"]).cuda(), sc["pose"], torch.from_numpy(sc["sem"]).cuda())
    compare_closed(to_np(m.extract()), oracle_map(w).extract(), "onehot")


def test_direct_batch_matches_oracle():
    """Direct per-pair reductions through slim_integrate_batch (all scans of
    two maps in shared grids) give the oracle's map."""
    from paper_2512_12945_gb300 import slim
    w = synth.street_lidar(n_scans=3, n_az=512)
    r = synth.room_lidar(n_scans=3)
    maps, items = [], []
    for wk in (w, r):
        m = slim.Map(voxel_size=wk.voxel_size, trunc=wk.trunc, num_classes=wk.num_classes,
                     min_range=wk.min_range, max_range=wk.max_range,
                     body_from_sensor=wk.body_from_sensor,
                     max_points=max(s["pts"].shape[0] for s in wk.scans), aggregation="direct")
        maps.append(m)
        for s in wk.scans:
            items.append((m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                          torch.from_numpy(s["sem"]).cuda()))
    slim.slim_integrate_batch(items)
    for m, wk in zip(maps, (w, r)):
        m.sync()
        compare_closed(to_np(m.extract()), oracle_map(wk).extract(), "onehot")


@pytest.mark.parametrize("batched", [False, True])
def test_latest_label_mode_matches_oracle(batched):
    """The non-Bayesian ablation (latest measurement wins): the label each
    voxel keeps is the oracle's last writer, bit for bit, whatever order the
    reductions run in; scans of one map in one batched launch keep their
    order through the scan stamp."""
    from paper_2512_12945_gb300 import slim
    w = synth.street_lidar(n_scans=4, n_az=512)
    if batched:
        m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="latest",
                     num_classes=w.num_classes, min_range=w.min_range, max_range=w.max_range,
                     body_from_sensor=w.body_from_sensor,
                     max_points=max(s["pts"].shape[0] for s in w.scans))
        slim.slim_integrate_batch([(m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                                    torch.from_numpy(s["sem"]).cuda()) for s in w.scans])
        m.sync()
    else:
        m = gpu_map(w, mode="latest")
    g = to_np(m.extract())
    o = oracle_map(w, mode="latest").extract()
    compare_closed(g, o, "onehot")
    with pytest.raises(slim.SlimError) as e:
        m.uncertainty()
    assert e.value.status == 6


@pytest.fixture(scope="module")
def _street100_oracle():
    w = synth.street_lidar(n_scans=100)
    return w, oracle_map(w).extract()


@pytest.mark.parametrize("agg", ["direct", "hash"])
def test_benchmark_configuration_full_parity(_street100_oracle, agg):
    """The benchmark's own configuration, compared in full: 100 street scans
    of 131,072 points through slim_integrate_batch (16 scans per launch),
    the map sized as the benchmark sizes it; every one of the ~1.95 M voxels
    matches the oracle (keys, weights and class counts bit for bit, D to
    FP32 rounding)."""
    from paper_2512_12945_gb300 import slim
    w, o = _street100_oracle
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
                 min_range=w.min_range, max_range=w.max_range,
                 body_from_sensor=w.body_from_sensor, block_capacity=65536,
                 hash_capacity=1 << 21, max_points=131072, aggregation=agg,
                 tile_points=256 if agg == "hash" else 0)
    slim.slim_integrate_batch([(m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                                torch.from_numpy(s["sem"]).cuda()) for s in w.scans])
    m.sync()
    g = to_np(m.extract())
    assert len(g["W"]) > 1_900_000
    compare_closed(g, o, "onehot")


@pytest.mark.parametrize("mode,agg", [("onehot", "direct"), ("onehot", "hash"),
                                      ("onehot", "sort"), ("latest", "auto")])
def test_max_classes_64(mode, agg):
    """K = 64 (the largest class count: the class index fills the 6 class
    bits of a hash-tile key and lives in the latest-label stamp's byte)."""
    w = synth.room_lidar(n_scans=3, K=64)
    g = to_np(gpu_map(w, mode=mode, aggregation=agg).extract())
    o = oracle_map(w, mode=mode).extract()
    compare_closed(g, o, "onehot")


def test_hash_table_full_is_a_capacity_fault():
    """A hash table too small for the scan's blocks: the probe limit raises
    SLIM_ERR_CAPACITY on the sticky status (nothing hangs), reset clears it."""
    from paper_2512_12945_gb300 import slim
    w = synth.street_lidar(n_scans=1, n_az=512)
    s = w.scans[0]
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=20, min_range=w.min_range,
                 max_range=w.max_range, body_from_sensor=w.body_from_sensor,
                 max_points=s["pts"].shape[0], hash_capacity=32)
    m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
    with pytest.raises(slim.SlimError) as e:
        m.sync()
    assert e.value.status == 3
    m.reset()
    m.sync()


@pytest.mark.parametrize("K", [10, 20, 7])
@pytest.mark.parametrize("agg", ["direct", "sort"])
def test_soft_counts_full_scans(K, agg):
    """Soft counts on full 64 x 2048 room scans, where a voxel collects
    hundreds of observations per scan (both strategies, including the batched
    direct grid). S, W and the class counts are 64-bit fixed-point sums
    (unit 2^-32, exact and independent of the order of the reductions), so D,
    W and every count meet the stated tolerance however many observations a
    voxel holds."""
    from paper_2512_12945_gb300 import slim
    w = synth.room_lidar(n_scans=3, n_beams=64, n_az=2048, K=K, mode="soft")
    o = oracle_map(w, mode="soft").extract()
    compare_closed(to_np(gpu_map(w, mode="soft", aggregation=agg).extract()), o, "soft")
    if agg == "direct":
        m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="soft", num_classes=K,
                     min_range=w.min_range, max_range=w.max_range, max_points=131072,
                     aggregation="direct")
        slim.slim_integrate_batch([(m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                                    torch.from_numpy(s["sem"]).cuda()) for s in w.scans])
        m.sync()
        compare_closed(to_np(m.extract()), o, "soft")



@pytest.mark.parametrize("mode,agg", [("onehot", "direct"), ("onehot", "hash"), ("onehot", "sort"),
                                      ("soft", "direct"), ("soft", "sort"), ("latest", "auto")])
def test_reset_leaves_no_stale_records(mode, agg):
    """The reset zeroes only the 2 x 2 x 2 sub-blocks each block marked as
    written. Integrate two scans, reset, integrate two other scans: the map
    must be the oracle's map of the second pair alone, for every record
    writer (direct reductions, hash tiles, sort tiles) and record layout."""
    import copy
    w = synth.street_lidar(n_scans=4, n_az=512)
    m = gpu_map(w, mode=mode, scans=w.scans[:2], aggregation=agg)
    m.reset()
    for s in w.scans[2:]:
        m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
    m.sync()
    w2 = copy.copy(w)
    w2.scans = w.scans[2:]
    o = oracle_map(w2, mode=mode).extract()
    compare_closed(to_np(m.extract()), o, "soft" if mode == "soft" else "onehot")
