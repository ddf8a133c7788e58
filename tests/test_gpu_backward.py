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


def _grads_closed(w, K, stored=False, mode="soft"):
    from paper_2512_12945_gb300 import autograd, slim
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode=mode, num_classes=K,
                 min_range=w.min_range, max_range=w.max_range,
                 body_from_sensor=w.body_from_sensor,
                 max_points=max(s["pts"].shape[0] for s in w.scans), block_capacity=200000,
                 hash_capacity=1 << 20)
    pts = [torch.from_numpy(s["pts"]).cuda().requires_grad_(True) for s in w.scans]
    sem = [torch.from_numpy(s["sem"]).cuda().requires_grad_(True) for s in w.scans]
    D, W, c, ijk = autograd.integrate(m, [s["pose"] for s in w.scans], pts, sem, stored=stored)
    rng = np.random.default_rng(5)
    a = torch.from_numpy(rng.standard_normal(D.shape[0]).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal(tuple(c.shape)).astype(np.float32)).cuda()
    loss = (a * D * D).sum() + (B * c).sum()
    loss.backward()
    gs = [s.grad.cpu().numpy() if s.grad is not None else np.zeros(s.shape, np.float32)
          for s in sem]
    return (D, c, ijk, a, B), [p.grad.cpu().numpy() for p in pts], gs


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


@pytest.mark.parametrize("mode", ["soft", "onehot"])
def test_stored_pair_list_gives_the_recomputed_gradients(mode):
    """The stored form of the reverse mode (slim_record_pairs, then
    slim_backward_pairs) runs the same per-pair terms in the same order as
    the recomputing one (slim_backward): on the same map and the same
    incoming gradients, the same results bit for bit, on full-size 64 x 2048
    room scans."""
    from paper_2512_12945_gb300 import slim
    w = synth.room_lidar(seed=4, n_scans=2, n_beams=64, n_az=2048, K=20, mode="soft")
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode=mode, num_classes=20,
                 min_range=w.min_range, max_range=w.max_range,
                 body_from_sensor=w.body_from_sensor,
                 max_points=max(s["pts"].shape[0] for s in w.scans), block_capacity=200000,
                 hash_capacity=1 << 20)
    data = [(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
            for s in w.scans]
    for p, pose, q in data:
        m.integrate(p, pose, q)
    idx = m.extract(index=True)["index"].long()
    size = int(idx.max().item()) + 1
    rng = np.random.default_rng(6)
    gD = torch.from_numpy(rng.standard_normal(size).astype(np.float32)).cuda()
    gS = torch.from_numpy(rng.standard_normal((size, 20)).astype(np.float32)).cuda()
    for p, pose, q in data:
        gs1, gx1 = m.backward(p, pose, q, gD, gS)
        offs, vox = m.record_pairs(p, pose)
        gs2, gx2 = m.backward_pairs(p, pose, offs, vox, gD, gS)
        assert torch.equal(gx1, gx2), (gx1 - gx2).abs().max().item()
        assert torch.equal(gs1, gs2)


def test_autograd_stored_form_soft():
    """autograd.integrate(..., stored=True) gives the gradients of the
    recomputing form (soft counts: the forward's sums are exact, so two maps
    built from the same scans are equal and so are the gradients)."""
    w = synth.room_lidar(seed=4, n_scans=2, n_beams=64, n_az=2048, K=20, mode="soft")
    (_, c1, ijk1, _, _), gp1, gs1 = _grads_closed(w, 20, stored=False)
    (_, c2, ijk2, _, _), gp2, gs2 = _grads_closed(w, 20, stored=True)
    assert torch.equal(ijk1, ijk2) and torch.equal(c1, c2)
    for k in range(len(w.scans)):
        assert np.array_equal(gp1[k], gp2[k]) and np.array_equal(gs1[k], gs2[k])


def test_stored_pair_list_layout():
    """The pair list is CSR by point: offsets rise by each point's pair
    count, the total is the number of the scan's kept observations (W summed
    over the voxels of a one-scan map), and every entry is a voxel of the
    map's extract index."""
    from paper_2512_12945_gb300 import slim
    w = synth.room_lidar(seed=4, n_scans=1, n_beams=16, n_az=512, K=20, mode="soft")
    s = w.scans[0]
    m = slim.Map(voxel_size=w.voxel_size, trunc=w.trunc, mode="soft", num_classes=20,
                 min_range=w.min_range, max_range=w.max_range,
                 body_from_sensor=w.body_from_sensor, max_points=s["pts"].shape[0])
    pts = torch.from_numpy(s["pts"]).cuda()
    m.integrate(pts, s["pose"], torch.from_numpy(s["sem"]).cuda())
    ext = m.extract(index=True)
    offs, vox = m.record_pairs(pts, s["pose"])
    o = offs.cpu().numpy().astype(np.int64)
    assert o[0] == 0 and np.all(np.diff(o) >= 0) and o[-1] == vox.numel()
    assert vox.numel() == int(round(float(ext["W"].sum())))
    assert set(np.unique(vox.cpu().numpy())) == set(ext["index"].cpu().numpy().tolist())
