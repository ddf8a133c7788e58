"""Batched integration: many maps of both kinds and uneven scan sizes in one
slim_integrate_batch call (closed-set scans in one persistent launch), eager
and captured in a CUDA graph, against per-map integration and the oracle."""
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
    for m, r in zip(maps[4:], refs[4:]):
        _compare_open(to_np(m.extract()), r)


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
