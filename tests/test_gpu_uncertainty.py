"""Uncertainty read-out against the oracle (which is pinned to scipy's
Dirichlet, entropy and Student-t routines): closed-set class-probability
variances and predictive entropy, open-set Student-t predictive variances."""
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


@pytest.mark.parametrize("mode,alpha0", [("onehot", 1.0), ("soft", 0.5), ("onehot", 0.0)])
def test_closed_uncertainty(mode, alpha0):
    w = synth.room_lidar(seed=1, n_scans=4, K=10, mode=mode)
    g = gpu_map(w, alpha0=alpha0)
    unc = g.uncertainty().cpu().numpy()
    o = oracle_map(w, alpha0=alpha0)
    ref = o.uncertainty()
    assert unc.shape == ref.shape
    assert np.array_equal(to_np(g.extract())["ijk"], o.extract()["ijk"])
    assert_close(unc, ref, 1e-4, 1e-7, "dirichlet variance / entropy")


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_open_uncertainty(storage):
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=64, height=48, dim=64, frames=[0, 1, 2])
    g = gpu_map(w, embed_storage=storage, voxel_capacity=200000)
    unc = g.uncertainty().cpu().numpy()
    ext = to_np(g.extract())
    o = oracle_map(w)
    ref = o.uncertainty()
    assert unc.shape == ref.shape
    inf = np.isinf(ref)
    assert np.array_equal(np.isinf(unc), inf)
    assert inf.any() and (~inf).any()
    if storage == "f32":
        assert_close(unc[~inf], ref[~inf], RTOL * 10, ATOL, "student-t variance")
    else:  # beta stored in BF16: a few half-ulps of 2^-9 per scan
        err = np.abs(unc[~inf] - ref[~inf])
        assert err.max() <= len(w.scans) * 2.0 ** -9 * np.abs(ref[~inf]).max() + 1e-6
    # the variance is the stated closed form of the stored beta and W
    W = ext["W"][:, None]
    closed = np.where(W > 2, 2.0 * ext["beta"] * (W + 1) / (W * np.maximum(W - 2, 1e-30)), np.inf)
    assert np.array_equal(np.isinf(closed), inf)
    assert_close(unc[~inf], closed[~inf], 1e-5, 1e-7, "closed form")
