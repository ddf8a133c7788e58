"""Batched integration: many maps of both kinds and uneven scan sizes in one
slim_integrate_batch call, eager and captured in a CUDA graph, against
per-map integration and against the oracle (every map, closed and open;
the 16-map configuration of the benchmark at full size included)."""
import numpy as np
import pytest

from paper_2512_12945_gb300 import synth
from helpers import RTOL, ATOL, assert_close, compare_closed, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _workloads():
    closed = [synth.street_lidar(seed=20 + k, n_scans=2, n_az=az)
              for k, az in enumerate((320, 700, 1300, 2048))]
    opened = [synth.indoor_rgbd(seed=30 + k, n_frames=40, width=w, height=h, dim=64,
                                frames=[0, 1])
              for k, (w, h) in enumerate(((48, 36), (64, 48), (80, 60), (96, 72)))]
    return closed, opened


def _maps(closed, opened):
    from paper_2512_12945_gb300 import slim
    maps = []
    for w in closed:
        maps.append(slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=20,
                             min_range=w.min_range, max_range=w.max_range,
                             body_from_sensor=w.body_from_sensor, max_points=131072,
                             block_capacity=100000, hash_capacity=1 << 18))
    for w in opened:
        maps.append(slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="open", embed_dim=64,
                             embed_storage="bf16", min_range=w.min_range, max_range=w.max_range,
                             max_points=w.scans[0]["pts"].shape[0], voxel_capacity=200000))
    return maps


def _items(maps, works):
    dev = []
    for m, w in zip(maps, works):
        for s in w.scans:
            dev.append((m, torch.from_numpy(s["pts"]).cuda(), s["pose"],
                        torch.from_numpy(s["sem"]).cuda()))
    return dev


def _compare_open(g, o):
    """BF16-stored means: two runs may sum a voxel's observations in another
    order, which can move a stored value by one BF16 ulp."""
    assert np.array_equal(g["ijk"], o["ijk"])
    assert np.array_equal(g["W"], o["W"])
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    for k in ("sem", "beta"):
        assert_close(g[k], o[k], 2.0 ** -7, 2.0 ** -9 * np.abs(o[k]).max(), k)


def _compare_open_oracle(g, o, n_scans):
    """BF16-stored means against the oracle's FP64 fusion: bit-exact key set
    and weights, D within the parity tolerance, and m and beta within one
    BF16 rounding per scan of the largest stored magnitude (half an ulp,
    2^-9, for m; beta's update also reads the rounded m: 2^-8)."""
    assert np.array_equal(g["ijk"], o["ijk"]), "voxel key sets differ"
    assert np.array_equal(g["W"].astype(np.float64), o["W"]), "weights differ"
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    for k, ulp in (("sem", 2.0 ** -9), ("beta", 2.0 ** -8)):
        err = np.abs(g[k] - o[k])
        assert err.max() <= n_scans * ulp * np.abs(o[k]).max() + 1e-6, (k, err.max())


def test_batch_matches_per_map_and_oracle():
    from paper_2512_12945_gb300 import slim
    closed, opened = _workloads()
    works = closed + opened
    ref_maps = _maps(closed, opened)
    for m, w in zip(ref_maps, works):
        for s in w.scans:
            m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"],
                        torch.from_numpy(s["sem"]).cuda())
    refs = [to_np(m.extract()) for m in ref_maps]
    maps = _maps(closed, opened)
    items = _items(maps, works)
    slim.slim_integrate_batch(items)
    for m, r, w in zip(maps[:4], refs[:4], closed):
        g = to_np(m.extract())
        compare_closed(g, r, "onehot")
        compare_closed(g, oracle_map(w).extract(), "onehot")
    for m, r, w in zip(maps[4:], refs[4:], opened):
        g = to_np(m.extract())
        _compare_open(g, r)
        _compare_open_oracle(g, oracle_map(w).extract(), len(w.scans))


def test_batch_full_16_maps_vs_oracle():
    """The benchmark's batched configuration at full size: 8 closed-set street
    maps (64 beams, 320-3900 azimuths, 20 classes) and 8 open-set RGB-D maps
    (l = 256, 320 x 240 to 640 x 480, BF16 storage), 10 scans each, all in
    one slim_integrate_batch call; every map against the oracle."""
    from paper_2512_12945_gb300 import slim
    closed, opened = synth.batch_workload(seed=5, n_scans=10)
    maps = []
    for w in closed:
        maps.append(slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=20,
                             min_range=w.min_range, max_range=w.max_range,
                             body_from_sensor=w.body_from_sensor,
                             max_points=max(s["pts"].shape[0] for s in w.scans),
                             block_capacity=200000, hash_capacity=1 << 19))
    for w in opened:
        maps.append(slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="open",
                             embed_dim=w.embed_dim, embed_storage="bf16",
                             min_range=w.min_range, max_range=w.max_range,
                             max_points=w.scans[0]["pts"].shape[0], voxel_capacity=400000,
                             image_width=w.image_width))
    items = _items(maps, closed + opened)
    slim.slim_integrate_batch(items)
    for m, w in zip(maps[:8], closed):
        compare_closed(to_np(m.extract()), oracle_map(w).extract(), "onehot")
    for m, w in zip(maps[8:], opened):
        _compare_open_oracle(to_np(m.extract()), oracle_map(w).extract(), len(w.scans))


def test_batch_in_cuda_graph():
    from paper_2512_12945_gb300 import slim
    closed, opened = _workloads()
    works = closed + opened
    maps = _maps(closed, opened)
    items = _items(maps, works)
    slim.slim_integrate_batch(items)  # eager, for reference
    refs = [to_np(m.extract()) for m in maps]
    for m in maps:
        m.reset()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for m in maps:
            m.reset()
        slim.slim_integrate_batch(items)
    for _ in range(2):  # replays start from empty maps
        graph.replay()
        torch.cuda.synchronize()
        for m, r in zip(maps[:4], refs[:4]):
            compare_closed(to_np(m.extract()), r, "onehot")
        for m, r in zip(maps[4:], refs[4:]):
            _compare_open(to_np(m.extract()), r)
