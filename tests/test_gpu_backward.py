"""Adjoint kernel (through torch.autograd) against the oracle's adjoint,
which the CPU tests pin to central finite differences of the forward pass."""
import numpy as np
import pytest

from paper_2512_12945_gb300 import synth
from helpers import oracle_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _close(g, o, what, rtol=1e-4):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    scale = max(np.abs(o).max(), 1e-12)
    err = np.abs(g - o)
    bad = err > rtol * np.abs(o) + 1e-5 * scale
    assert not bad.any(), (what, int(bad.sum()), bad.size, err.max(), scale)


def _grads_closed(w, K):
    from paper_2512_12945_gb300 import autograd, slim
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="soft", num_classes=K,
                 min_range=w.min_range, max_range=w.max_range,
                 body_from_sensor=w.body_from_sensor,
                 max_points=max(s["pts"].shape[0] for s in w.scans), block_capacity=200000,
                 hash_capacity=1 << 20)
    pts = [torch.from_numpy(s["pts"]).cuda().requires_grad_(True) for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda().requires_grad_(True) for s in w.scans]
    D, W, c, ijk = autograd.integrate(m, [s["pose"] for s in w.scans], pts, sem)
    rng = np.random.default_rng(5)
    a = torch.from_numpy(rng.standard_normal(D.shape[0]).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal(tuple(c.shape)).astype(np.float32)).cuda()
    loss = (a * D * D).sum() + (B * c).sum()
    loss.backward()
    return (D, c, ijk, a, B), [p.grad.cpu().numpy() for p in pts], [s.grad.cpu().numpy() for s in sem]


def test_closed_soft_gradients_match_oracle():
    w = synth.room_lidar(n_scans=3, n_beams=16, n_az=256, K=10, mode="soft")
    (D, c, ijk, a, B), gp, gs = _grads_closed(w, 10)
    om = oracle_map(w, mode="soft")
    o = om.extract()
    assert np.array_equal(ijk.cpu().numpy(), o["ijk"])
    gD = 2 * a.cpu().numpy().astype(np.float64) * o["D"]
    gS = B.cpu().numpy().astype(np.float64)
    for k, s in enumerate(w.scans):
        ogs, ogx = om.backward_scan(s["pts"], s["pose"], s["sem"], gD, gS)
        _close(gs[k], ogs, f"dL/dp scan {k}")
        _close(gp[k], ogx, f"dL/dxyz scan {k}", rtol=2e-3)


def test_closed_soft_full_size_scan():
    """Full 64 x 2048 scans (the differentiation workload's sensor)."""
    w = synth.room_lidar(n_scans=2, n_beams=64, n_az=2048, K=20, mode="soft")
    (D, c, ijk, a, B), gp, gs = _grads_closed(w, 20)
    om = oracle_map(w, mode="soft")
    o = om.extract()
    assert np.array_equal(ijk.cpu().numpy(), o["ijk"])
    gD = 2 * a.cpu().numpy().astype(np.float64) * o["D"]
    s = w.scans[1]
    ogs, ogx = om.backward_scan(s["pts"], s["pose"], s["sem"], gD, B.cpu().numpy())
    _close(gs[1], ogs, "dL/dp")
    _close(gp[1], ogx, "dL/dxyz", rtol=2e-3)


def test_open_gradients_match_oracle():
    from paper_2512_12945_gb300 import autograd, slim
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=48, height=36, dim=64, frames=[0, 1])
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="open", embed_dim=64,
                 min_range=w.min_range, max_range=w.max_range,
                 max_points=w.scans[0]["pts"].shape[0], voxel_capacity=100000)
    pts = [torch.from_numpy(s["pts"]).cuda().requires_grad_(True) for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda().requires_grad_(True) for s in w.scans]
    D, W, mm, beta, ijk = autograd.integrate(m, [s["pose"] for s in w.scans], pts, sem)
    rng = np.random.default_rng(6)
    A = torch.from_numpy(rng.standard_normal(tuple(mm.shape)).astype(np.float32)).cuda()
    Bq = torch.from_numpy(rng.standard_normal(tuple(beta.shape)).astype(np.float32)).cuda()
    loss = (A * mm * mm).sum() + (Bq * beta).sum() + (D * D).sum()
    loss.backward()
    om = oracle_map(w)
    o = om.extract()
    assert np.array_equal(ijk.cpu().numpy(), o["ijk"])
    gS = 2 * A.cpu().numpy().astype(np.float64) * o["sem"]
    gD = 2 * o["D"]
    for k, s in enumerate(w.scans):
        ogs, ogx = om.backward_scan(s["pts"], s["pose"], s["sem"], gD, gS, Bq.cpu().numpy())
        _close(sem[k].grad.cpu().numpy(), ogs, f"dL/dz scan {k}", rtol=1e-3)
        _close(pts[k].grad.cpu().numpy(), ogx, f"dL/dxyz scan {k}", rtol=2e-3)
