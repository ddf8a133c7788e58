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
    w = _work(frames=3)
    z = np.random.default_rng(0).standard_normal(64).astype(np.float32)
    for s in w.scans:
        s["sem"] = np.ascontiguousarray(np.tile(z, (s["pts"].shape[0], 1)))
    g = to_np(gpu_map(w, voxel_capacity=200000).extract())
    assert np.abs(g["beta"]).max() < 1e-6
    assert_close(g["sem"], np.tile(z, (len(g["W"]), 1)), 1e-6, 1e-6, "m")


def test_open_voxel_capacity_fault():
    from paper_2512_12945_gb300 import slim
    w = _work(frames=1)
    with pytest.raises(slim.SlimError) as e:
        gpu_map(w, voxel_capacity=10)
    assert e.value.status == 3


def test_open_long_runs_split_across_pieces():
    """Full-resolution depth frames where single voxels collect thousands of
    pixel observations in one frame (the camera close to a wall): runs far
    longer than one piece of sorted pairs are cut and merged, and must give
    the same batch update as the oracle's sequential one."""
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
