"""Parity of the weighted TSDF update (w~ of Sec. III-A, the linear decay
behind the surface) against the oracle: identical voxel sets, FP32 W, D and
class counts within 1e-5 relative / 1e-6 absolute (the weights are no longer
integers, so W and the counts are FP32 sums of per-observation weights,
accumulated in any order)."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import RTOL, ATOL, assert_close, gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _compare(g, o, mode):
    assert np.array_equal(g["ijk"], o["ijk"]), "voxel key sets differ"
    assert_close(g["W"], o["W"], RTOL, ATOL, "W")
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    if mode == "latest":
        assert np.array_equal(g["sem"].astype(np.float64), o["sem"]), "labels differ"
    else:
        assert_close(g["sem"], o["sem"], RTOL, ATOL, "counts")
        assert_close(g["sem"].sum(1), g["W"], RTOL, ATOL, "sum c = W")


@pytest.mark.parametrize("mode", ["onehot", "soft", "latest"])
def test_weighted_room_matches_oracle(mode):
    w = synth.room_lidar(n_scans=6)
    g = to_np(gpu_map(w, mode=mode, weighting="linear", weight_eps=EPS).extract())
    o = oracle_map(w, mode=mode, weighting=1, weight_eps=EPS).extract()
    _compare(g, o, mode)
    # the behind-surface voxels carry less weight than in the w~ = 1 map
    u = oracle_map(w, mode=mode).extract()
    assert o["W"].sum() < u["W"].sum()


def test_weighted_and_unweighted_maps_in_one_batch():
    """A weighted and an unweighted map integrated by one slim_integrate_batch
    call (their scans run in separate grids) each match their oracle."""
    from paper_2512_12945_gb300 import slim
    w = synth.street_lidar(n_scans=3, n_az=512)
    kw = dict(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=w.num_classes,
              min_range=w.min_range, max_range=w.max_range, body_from_sensor=w.body_from_sensor,
              max_points=max(s["pts"].shape[0] for s in w.scans))
    mw = slim.Map(weighting="linear", weight_eps=EPS, **kw)
    mu = slim.Map(**kw)
    items = []
    for s in w.scans:
        p = torch.from_numpy(s["pts"]).cuda()
        q = torch.from_numpy(s["sem"]).cuda()
        items += [(mw, p, s["pose"], q), (mu, p, s["pose"], q)]
    slim.slim_integrate_batch(items)
    mw.sync()
    mu.sync()
    _compare(to_np(mw.extract()), oracle_map(w, weighting=1, weight_eps=EPS).extract(), "onehot")
    gu, ou = to_np(mu.extract()), oracle_map(w).extract()
    assert np.array_equal(gu["ijk"], ou["ijk"])
    assert np.array_equal(gu["W"].astype(np.float64), ou["W"])


def test_weighting_argument_checks():
    from paper_2512_12945_gb300 import slim
    with pytest.raises(slim.SlimError) as e:
        slim.Map(mode="open", embed_dim=64, weighting="linear", weight_eps=EPS)
    assert e.value.status == 1
    with pytest.raises(slim.SlimError) as e:
        slim.Map(aggregation="hash", weighting="linear", weight_eps=EPS)
    assert e.value.status == 1
    with pytest.raises(slim.SlimError) as e:
        slim.Map(trunc=0.3, weighting="linear", weight_eps=0.3)
    assert e.value.status == 1
    w = synth.room_lidar(n_scans=1, n_beams=8, n_az=64)
    m = gpu_map(w, mode="soft", weighting="linear", weight_eps=EPS)
    ext = m.extract()
    n = len(ext["W"])
    s = w.scans[0]
    with pytest.raises(slim.SlimError) as e:
        m.backward(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda(),
                   torch.zeros(n, device="cuda"), torch.zeros((n, w.num_classes), device="cuda"))
    assert e.value.status == 6
