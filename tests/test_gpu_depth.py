"""RGB-D front end (slim_integrate_depth): depth frames back-projected inside
the traversal kernels give the oracle's map for the same frames (the oracle
back-projects in the same FP32 order, pinned against numpy), in the open set
and the closed-set modes."""
import numpy as np
import pytest

from paper_2512_12945_gb300 import synth
from helpers import RTOL, ATOL, assert_close, compare_closed, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _frames(W=96, H=72, dim=64, n=3):
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=W, height=H, dim=dim, frames=list(range(n)))
    f = np.float32(525.0 * W / 640.0)
    out = []
    for s in w.scans:
        depth = s["pts"][:, 2].reshape(H, W).astype(np.float32).copy()
        depth[depth <= 0] = 0.0
        out.append((depth, s))
    return w, out, f, np.float32(W / 2), np.float32(H / 2)


def _maps(w, frames, f, cx, cy, mode, sem_of, **kw):
    import oracle
    from paper_2512_12945_gb300 import slim
    H, W = frames[0][0].shape
    width = w.embed_dim if mode == "open" else 10
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode=mode, num_classes=10,
                 embed_dim=w.embed_dim, min_range=w.min_range, max_range=w.max_range,
                 max_points=H * W, **kw)
    code = {"onehot": oracle.CLOSED_ONEHOT, "soft": oracle.CLOSED_SOFT, "open": oracle.OPEN,
            "latest": oracle.CLOSED_LATEST}[mode]
    o = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, mode=code, num_classes=10,
                         embed_dim=w.embed_dim, min_range=w.min_range, max_range=w.max_range)
    for depth, s in frames:
        sem = sem_of(s).astype(np.float32)
        m.integrate_depth(torch.from_numpy(depth).cuda(), f, f, cx, cy, s["pose"],
                          torch.from_numpy(np.ascontiguousarray(sem)).cuda())
        o.integrate_depth(depth, f, f, cx, cy, s["pose"], sem)
    m.sync()
    assert width == m.width
    return to_np(m.extract()), o.extract()


def test_depth_open_set():
    w, frames, f, cx, cy = _frames()
    g, o = _maps(w, frames, f, cx, cy, "open", lambda s: s["sem"], voxel_capacity=400000)
    assert np.array_equal(g["ijk"], o["ijk"])
    assert np.array_equal(g["W"].astype(np.float64), o["W"])
    assert_close(g["D"], o["D"], RTOL, ATOL, "D")
    assert_close(g["sem"], o["sem"], RTOL, ATOL, "m")
    assert_close(g["beta"], o["beta"], RTOL, ATOL, "beta")


@pytest.mark.parametrize("mode", ["onehot", "soft", "latest"])
def test_depth_closed_modes(mode):
    w, frames, f, cx, cy = _frames()
    rng = np.random.default_rng(9)

    def probs(s):
        return synth.dirichlet_probs(rng, s["labels"] % 10, 10)

    # the same probabilities on both sides: draw them once per frame
    frames = [(d, dict(s, sem10=probs(s))) for d, s in frames]
    g, o = _maps(w, frames, f, cx, cy, mode, lambda s: s["sem10"])
    compare_closed(g, o, "soft" if mode == "soft" else "onehot")
