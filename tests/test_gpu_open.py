"""Open-set parity of the CUDA path against the oracle: bit-exact voxel sets
and weights; FP32-stored NIG mean m and beta, and D, within 1e-5 relative /
1e-6 absolute; BF16 storage against the FP64 oracle within its stated bound."""
import numpy as np
import pytest

from paper_2512_12945_gb300 import synth
from helpers import RTOL, ATOL, assert_close, gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _work(frames=4, w=64, h=48, dim=64, seed=3):
    return synth.indoor_rgbd(seed=seed, n_frames=40, width=w, height=h, dim=dim,
                             frames=list(range(frames)))


def _compare(g, o, rtol=RTOL, atol=ATOL, sem_tol=None):
    assert np.array_equal(g["ijk"], o["ijk"]), "voxel key sets differ"
    assert np.array_equal(g["W"].astype(np.float64), o["W"]), "weights differ"
    assert_close(g["D"], o["D"], rtol, atol, "D")
    st = sem_tol or (rtol, atol)
    assert_close(g["sem"], o["sem"], st[0], st[1], "m")
    assert_close(g["beta"], o["beta"], st[0], st[1], "beta")


def test_open_fp32_parity():
    w = _work()
    g = to_np(gpu_map(w, voxel_capacity=200000).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_fp32_dim512_full_width_frames():
    w = _work(frames=2, w=160, h=120, dim=512)
    g = to_np(gpu_map(w, voxel_capacity=300000).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_bf16_storage_error_bound():
    """m and beta stored in BF16 (8-bit mantissa), accumulated in FP32: each
    stored value carries at most half a BF16 ulp of rounding per scan."""
    w = _work(frames=4)
    g = to_np(gpu_map(w, embed_storage="bf16", voxel_capacity=200000).extract())
    o = oracle_map(w).extract()
    assert np.array_equal(g["ijk"], o["ijk"])
    assert np.array_equal(g["W"].astype(np.float64), o["W"])
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    # one BF16 rounding (half an ulp, 2^-9 relative) per scan of a value whose
    # magnitude along the way is bounded by the largest stored magnitude
    n = len(w.scans)
    for k in ("sem", "beta"):
        scale = np.abs(o[k]).max()
        err = np.abs(g[k] - o[k])
        assert err.max() <= n * 2.0 ** -9 * scale + 1e-6, (k, err.max(), scale)


def test_open_ragged_and_empty():
    w = _work(frames=2)
    s0 = w.scans[0]
    w.scans = [dict(pts=s0["pts"][:0], pose=s0["pose"], sem=s0["sem"][:0]),
               dict(pts=s0["pts"][:1001], pose=s0["pose"], sem=s0["sem"][:1001]),
               w.scans[1]]
    g = to_np(gpu_map(w, voxel_capacity=100000).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_identical_embeddings_give_zero_beta():
    """Identical (not normalised) embeddings: beta stays 0 and m = z; the
    map's embed_bound covers their largest element."""
    w = _work(frames=3)
    z = np.random.default_rng(0).standard_normal(64).astype(np.float32)
    for s in w.scans:
        s["sem"] = np.ascontiguousarray(np.tile(z, (s["pts"].shape[0], 1)))
    g = to_np(gpu_map(w, voxel_capacity=200000, embed_bound=4.0).extract())
    assert np.abs(g["beta"]).max() < 1e-6
    assert_close(g["sem"], np.tile(z, (len(g["W"]), 1)), 1e-6, 1e-6, "m")


def test_open_embedding_beyond_bound_raises_range():
    """An embedding element beyond the map's embed_bound (here 10 against
    the default bound 1) is reported as SLIM_ERR_RANGE; the same scans under
    a bound that covers them match the oracle."""
    from paper_2512_12945_gb300 import slim
    w = _work(frames=2)
    for s in w.scans:
        s["sem"] = np.ascontiguousarray(s["sem"] * 10.0, dtype=np.float32)
    with pytest.raises(slim.SlimError) as e:
        gpu_map(w, voxel_capacity=200000)
    assert e.value.status == 8
    g = to_np(gpu_map(w, voxel_capacity=200000, embed_bound=16.0).extract())
    _compare(g, oracle_map(w).extract())


def test_open_voxel_capacity_fault():
    from paper_2512_12945_gb300 import slim
    w = _work(frames=1)
    with pytest.raises(slim.SlimError) as e:
        gpu_map(w, voxel_capacity=10)
    assert e.value.status == 3


def test_open_long_runs_many_tiles():
    """Full-resolution depth frames where single voxels collect thousands of
    pixel observations in one frame (the camera close to a wall), summed by
    many tiles into one accumulator: the same update as the oracle's
    sequential one."""
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=64,
                          frames=[100, 0, 50])
    g = to_np(gpu_map(w, voxel_capacity=400000).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_max_dim_1024_bf16():
    """l = 1024 (the largest embedding: 8 element chunks per pass loop) with
    BF16 storage, against the oracle. Each scan rounds m and beta to BF16
    (half an ulp each, 2^-9 relative); the next scan's beta update uses the
    rounded m, which moves beta by another rounding of the same order, so
    beta is bounded by one ulp (2^-8) of its largest magnitude per scan and
    m by half an ulp per scan."""
    w = _work(frames=2, w=48, h=36, dim=1024)
    g = to_np(gpu_map(w, embed_storage="bf16", voxel_capacity=100000).extract())
    o = oracle_map(w).extract()
    assert np.array_equal(g["ijk"], o["ijk"])
    assert np.array_equal(g["W"].astype(np.float64), o["W"])
    n = len(w.scans)
    for k, ulp in (("sem", 2.0 ** -9), ("beta", 2.0 ** -8)):
        err = np.abs(g[k] - o[k])
        assert err.max() <= n * ulp * np.abs(o[k]).max() + 1e-6, k


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_open_full_frames_640x480_dim512(storage):
    """The indoor benchmark's frames at full size: 640 x 480 pixels, l = 512,
    both storages, against the oracle (FP32: the parity tolerance; BF16: one
    storage rounding per scan, as in test_open_bf16_storage_error_bound)."""
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=640, height=480, dim=512,
                          frames=[0, 7])
    g = to_np(gpu_map(w, embed_storage=storage, voxel_capacity=400000).extract())
    o = oracle_map(w).extract()
    if storage == "f32":
        _compare(g, o)
        return
    assert np.array_equal(g["ijk"], o["ijk"])
    assert np.array_equal(g["W"].astype(np.float64), o["W"])
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    n = len(w.scans)
    for k, ulp in (("sem", 2.0 ** -9), ("beta", 2.0 ** -8)):
        err = np.abs(g[k] - o[k])
        assert err.max() <= n * ulp * np.abs(o[k]).max() + 1e-6, (k, err.max())


def test_open_unorganized_points():
    """The same frames passed as unorganized points (tiles of 256
    consecutive points instead of 16 x 16 pixels): the tiling changes how
    observations are grouped, not the result."""
    w = _work(frames=3, w=160, h=120, dim=64)
    g = to_np(gpu_map(w, voxel_capacity=200000, image_width=0).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_tile_overflow_splits():
    """Scattered points (random directions and ranges, wide band): 256
    consecutive points touch thousands of distinct voxels, more than a
    tile's tables hold, so every tile is split into smaller pixel ranges
    until each fits; the result is unchanged."""
    rng = np.random.default_rng(7)
    n = 3000
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = (d * rng.uniform(0.5, 3.0, (n, 1))).astype(np.float32)
    z = rng.standard_normal((n, 64))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    w = _work(frames=1)
    w.trunc = 4 * w.voxel_size  # the widest band: 27 voxels per point
    w.image_width = 0
    w.scans = [dict(pts=pts, pose=np.eye(4), sem=z.astype(np.float32)),
               dict(pts=pts[::-1].copy(), pose=np.eye(4), sem=z[::-1].astype(np.float32).copy())]
    g = to_np(gpu_map(w, voxel_capacity=400000, block_capacity=100000).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


@pytest.mark.parametrize("tile_w", [8, 32])
def test_open_tile_shapes(tile_w):
    """Tiles of 8 x 32 and 32 x 8 pixels (the autotuner's other candidates):
    same result as the oracle."""
    w = _work(frames=3, w=160, h=120, dim=64)
    g = to_np(gpu_map(w, voxel_capacity=200000, tile_points=tile_w).extract())
    o = oracle_map(w).extract()
    _compare(g, o)


def test_open_autotune_picks_a_tile_shape():
    from paper_2512_12945_gb300 import slim
    w = _work(frames=2, w=320, h=240, dim=128)
    m = gpu_map(w, scans=[], voxel_capacity=200000)
    s = w.scans[0]
    best = m.autotune(torch.from_numpy(s["pts"]).cuda(), s["pose"],
                      torch.from_numpy(s["sem"]).cuda())
    assert best in (8, 16, 32)
    assert m.stats()["voxels"] == 0  # the map is left empty
    for s in w.scans:
        m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
    _compare(to_np(m.extract()), oracle_map(w).extract())
    u = gpu_map(w, scans=[], voxel_capacity=200000, image_width=0)
    assert u.autotune(torch.from_numpy(s["pts"]).cuda(), s["pose"],
                      torch.from_numpy(s["sem"]).cuda()) == 0


def test_open_host_entry_point():
    """slim_integrate_host for the open set (embeddings copied from pinned
    host memory into the map's staging buffers): the oracle's map."""
    from paper_2512_12945_gb300 import slim
    w = _work(frames=4, w=96, h=72, dim=64)
    m = gpu_map(w, scans=[], voxel_capacity=200000)
    host = [(torch.from_numpy(s["pts"]).pin_memory(), torch.from_numpy(s["sem"]).pin_memory())
            for s in w.scans]
    for (p, q), s in zip(host, w.scans):
        m.integrate_host(p, s["pose"], q)
    m.sync()
    _compare(to_np(m.extract()), oracle_map(w).extract())
