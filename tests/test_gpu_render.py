"""Ray-cast render (slim_render) against the oracle's renderer (pinned by
brute-force traversal and a plane's closed-form depth): same surface voxel
per pixel, the same label, depth and query cosine to FP32 rounding. Where
the two differ (a hit against a miss, or another crossing voxel), the pixel
is checked to be a sign tie: along that pixel's ray (the oracle's
traversal), each renderer's crossing must be the first crossing of its own
map's D values, and every voxel where the two maps disagree on the sign of D
must hold an oracle D within the parity tolerance of 0 (several answers are
then correct)."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import ATOL, RTOL, gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I32MIN = np.iinfo(np.int32).min


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _cam(o, forward="x"):
    T = np.eye(4)
    if forward == "x":  # camera z -> world x, camera x -> world -y, camera y -> world -z
        T[:3, :3] = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    else:  # looking along +y
        T[:3, :3] = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]])
    T[:3, 3] = o
    return T


def _first_crossing(vis, D):
    """Index in vis of the first voxel entered right after a visited voxel
    that is also in the map, with D_prev > 0 >= D (None if none)."""
    prev = None
    for k, ijk in enumerate(vis):
        d = D.get(tuple(ijk))
        if d is None:
            prev = None
            continue
        if prev is not None and prev > 0.0 and d <= 0.0:
            return k
        prev = d
    return None


def _compare(g, o, sim=False, maps=None, cam=None):
    """maps = (gpu extract, oracle extract, voxel size) and cam = the render
    arguments enable
    the tie check of the pixels where the two renderers differ."""
    gd, od = g["depth"].cpu().numpy(), o["depth"]
    gi, oi = g["ijk"].cpu().numpy(), o["ijk"]
    ghit, ohit = np.isfinite(gd), np.isfinite(od)
    assert ohit.sum() > 0.2 * ohit.size
    both = ghit & ohit
    same = both & (gi == oi).all(-1)
    differ = ~same & (ghit | ohit)
    assert differ.mean() < 0.01
    np.testing.assert_allclose(gd[same], od[same], rtol=1e-4, atol=1e-4)
    assert (gi[~ghit] == I32MIN).all()
    assert np.array_equal(g["label"].cpu().numpy()[same], o["label"][same])
    if sim:
        np.testing.assert_allclose(g["sim"].cpu().numpy()[same], o["sim"][same], atol=1e-4)
    if maps is None:
        return
    ge, oe, voxel_size = maps
    Dg = {tuple(k): float(d) for k, d in zip(ge["ijk"], ge["D"])}
    Do = {tuple(k): float(d) for k, d in zip(oe["ijk"], oe["D"])}
    assert Dg.keys() == Do.keys()
    T, fx, fy, cx, cy, width, height, near, far = cam
    for pix in np.flatnonzero(differ.ravel()):
        py, px = divmod(int(pix), width)
        vis = oracle.pixel_visits(voxel_size, T, fx, fy, cx, cy, px, py, near, far)
        kg, ko = _first_crossing(vis, Dg), _first_crossing(vis, Do)
        exp_g = tuple(vis[kg]) if kg is not None else None
        exp_o = tuple(vis[ko]) if ko is not None else None
        got_g = tuple(gi.reshape(-1, 3)[pix]) if ghit.ravel()[pix] else None
        got_o = tuple(oi.reshape(-1, 3)[pix]) if ohit.ravel()[pix] else None
        assert got_g == exp_g and got_o == exp_o, (pix, got_g, exp_g, got_o, exp_o)
        end = max(k for k in (kg, ko, len(vis) - 1) if k is not None)
        ties = 0
        for ijk in vis[:end + 1]:
            key = tuple(ijk)
            if key not in Do:
                continue
            if (Dg[key] > 0.0) != (Do[key] > 0.0):
                assert abs(Dg[key] - Do[key]) <= ATOL + RTOL * abs(Do[key]), (pix, key)
                assert abs(Do[key]) <= ATOL + RTOL * abs(Do[key]), (pix, key, Do[key])
                ties += 1
        assert ties > 0, pix


def test_render_closed_street():
    w = synth.street_lidar(n_scans=4, n_az=1024)
    m = gpu_map(w)
    om = oracle_map(w)
    maps = (to_np(m.extract()), om.extract(), w.voxel_size)
    T = _cam([3.0, 0.0, 1.6])
    args = (T, 100.0, 100.0, 80.0, 60.0, 160, 120, 0.5, 60.0)
    _compare(m.render(*args), om.render(*args), maps=maps, cam=args)
    T2 = _cam([2.0, -1.0, 1.6], "y")
    args = (T2, 120.0, 120.0, 64.0, 48.0, 128, 96, 0.2, 40.0)
    _compare(m.render(*args), om.render(*args), maps=maps, cam=args)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_render_open_query_cosine(storage):
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=96, height=72, dim=64, frames=[0, 1, 2])
    m = gpu_map(w, embed_storage=storage, voxel_capacity=400000)
    om = oracle_map(w)
    q = synth.random_queries(5, 1, 64)[0]
    T = w.scans[1]["pose"]
    args = (T, 60.0, 60.0, 48.0, 36.0, 96, 72, 0.3, 8.0)
    g = m.render(*args, q=torch.from_numpy(q).cuda())
    o = om.render(*args, q=q)
    maps = (to_np(m.extract()), om.extract(), w.voxel_size)
    if storage == "f32":
        _compare(g, o, sim=True, maps=maps, cam=args)
    else:  # BF16 means: the cosine within the BF16 rounding of m
        _compare(g, o, sim=False, maps=maps, cam=args)
        gs, os_ = g["sim"].cpu().numpy(), o["sim"]
        same = np.isfinite(o["depth"]) & (g["ijk"].cpu().numpy() == o["ijk"]).all(-1)
        assert np.abs(gs[same] - os_[same]).max() < 2e-2


def test_render_empty_map_and_bad_args():
    from paper_2512_12945_gb300 import slim
    w = synth.room_lidar(n_scans=1)
    m = gpu_map(w, scans=[])
    out = m.render(_cam([5.0, 5.0, 1.5]), 50.0, 50.0, 16.0, 12.0, 32, 24, 0.1, 20.0)
    assert torch.isinf(out["depth"]).all()
    assert (out["label"] == -1).all()
    for bad in [dict(width=0), dict(near=-1.0), dict(far=0.05), dict(fx=0.0)]:
        kw = dict(world_from_camera=_cam([5.0, 5.0, 1.5]), fx=50.0, fy=50.0, cx=16.0, cy=12.0,
                  width=32, height=24, near=0.1, far=20.0)
        kw.update(bad)
        with pytest.raises(slim.SlimError) as e:
            m.render(**kw)
        assert e.value.status == 1


def test_render_latest_label_map():
    w = synth.street_lidar(n_scans=3, n_az=1024)
    m = gpu_map(w, mode="latest")
    om = oracle_map(w, mode="latest")
    args = (_cam([3.0, 0.0, 1.6]), 100.0, 100.0, 80.0, 60.0, 160, 120, 0.5, 60.0)
    _compare(m.render(*args), om.render(*args),
             maps=(to_np(m.extract()), om.extract(), w.voxel_size), cam=args)
