"""Pins of the oracle against facts that do not come from the oracle itself:
a hand-derived worked example, closed forms, brute force on tiny grids, the
theorems' batch forms, invariants and finite differences (CPU only)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
V, TAU = 0.1, 0.3


def _pose_t(x, y, z):
    m = np.eye(4)
    m[:3, 3] = (x, y, z)
    return m


def _rand_pose(rng, spread=0.3):
    a = rng.uniform(0, 2 * math.pi, 3)
    cx, sx = math.cos(a[0]), math.sin(a[0])
    cy, sy = math.cos(a[1]), math.sin(a[1])
    cz, sz = math.cos(a[2]), math.sin(a[2])
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    m = np.eye(4)
    m[:3, :3] = Rz @ Ry @ Rx
    m[:3, 3] = rng.uniform(-spread, spread, 3)
    return m


def _onehot_probs(labels, K):
    p = np.full((len(labels), K), 0.05, np.float32)
    p[np.arange(len(labels)), labels] = 0.6
    return p


# ------------------------------------------------------------- worked example
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "axis_two_scans.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_worked_example_closed():
    g = _golden_rows()
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=4, alpha0=1.0)
    o = _pose_t(0.05, 0.05, 0.05)
    m.integrate([[1.02, 0, 0]], o, _onehot_probs(np.array([1]), 4))
    m.integrate([[1.04, 0, 0]], o, _onehot_probs(np.array([2]), 4))
    e = m.extract()
    assert np.array_equal(e["ijk"], g[:, :3].astype(np.int32))
    assert np.array_equal(e["W"], g[:, 3])
    np.testing.assert_allclose(e["D"], g[:, 4], atol=1e-6)
    assert np.array_equal(e["sem"], np.tile([0.0, 1.0, 1.0, 0.0], (7, 1)))
    post = m.extract(posterior=True)["sem"]
    np.testing.assert_allclose(post, np.tile([1 / 6, 2 / 6, 2 / 6, 1 / 6], (7, 1)), rtol=1e-15)


def test_worked_example_open():
    g = _golden_rows()
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, mode=oracle.OPEN, embed_dim=2)
    o = _pose_t(0.05, 0.05, 0.05)
    m.integrate([[1.02, 0, 0]], o, [[1.0, 0.0]])
    m.integrate([[1.04, 0, 0]], o, [[0.0, 1.0]])
    e = m.extract()
    assert np.array_equal(e["ijk"], g[:, :3].astype(np.int32))
    np.testing.assert_allclose(e["D"], g[:, 4], atol=1e-6)
    np.testing.assert_allclose(e["sem"], 0.5, rtol=1e-15)
    np.testing.assert_allclose(e["beta"], 0.25, rtol=1e-15)


def test_worked_example_query():
    # two orthogonal queries, voxel mean (0.8, 0.6): cosines (0.8, 0.6),
    # softmax of cos / 0.1 -> p0 = 1 / (1 + e^-2)
    label, prob, cos = oracle.query(np.array([[0.8, 0.6], [0.0, 0.0]]),
                                    np.array([[1, 0], [0, 1]], np.float32), 0.1, 0.1)
    assert label.tolist() == [0, -1]
    assert prob[0] == pytest.approx(1.0 / (1.0 + math.exp(-2.0)), rel=1e-14)
    assert prob[1] == 0.0
    np.testing.assert_allclose(cos[0], [0.8, 0.6], rtol=1e-14)
    # threshold: 256 equal cosines give p = 1/256 < 0.1 -> rejected
    q = np.tile(np.array([[1.0, 0.0]], np.float32), (256, 1))
    label, prob, _ = oracle.query(np.array([[3.0, 0.0]]), q, 0.01, 0.1)
    assert label[0] == -1 and prob[0] == pytest.approx(1 / 256)


# --------------------------------------------------------------- geometry pins
def test_axis_ray_closed_form():
    """A ray along +x: the voxels are the x-run covering the band and
    d = x_0 - c exactly (FP32 rounding only)."""
    p = oracle.make_params(V, TAU)
    o = _pose_t(0.05, 0.05, 0.05)
    for r in [0.517, 1.3337, 2.71, 7.77, 12.345]:
        vis = oracle.point_visits(p, [r, 0, 0], o)
        x0 = 0.05 + r
        lo = math.floor((x0 - TAU) / V)
        hi = math.floor((x0 + TAU) / V)
        assert vis[:, 0].tolist() == list(range(lo, hi + 1))
        assert (vis[:, 1:] == 0).all()
        ijk, pt, d = oracle.scan_pairs(p, np.array([[r, 0, 0]]), o)
        c = (ijk[:, 0] + 0.5) * V
        ref = np.minimum(x0 - c, TAU)
        keep = (x0 - (np.arange(lo, hi + 1) + 0.5) * V) >= -TAU
        assert len(d) == keep.sum()
        np.testing.assert_allclose(d, ref, atol=2e-6)


def _segment_cells_fp64(o, x, tau, v, margin):
    """Cells whose box meets the segment o + t u, t in [max(0, r - tau), r + tau],
    by brute force over the segment's bounding box. Returns (set, ambiguous)."""
    dl = x - o
    r = np.linalg.norm(dl)
    u = dl / r
    t0, t1 = max(0.0, r - tau), r + tau
    a, b = o + t0 * u, o + t1 * u
    lo = np.floor(np.minimum(a, b) / v).astype(int) - 1
    hi = np.floor(np.maximum(a, b) / v).astype(int) + 1
    cells, amb = set(), False
    for i in range(lo[0], hi[0] + 1):
        for j in range(lo[1], hi[1] + 1):
            for k in range(lo[2], hi[2] + 1):
                cmin = np.array([i, j, k]) * v
                cmax = cmin + v
                tin, tout = t0, t1
                for ax in range(3):
                    if abs(u[ax]) < 1e-300:
                        if not (cmin[ax] <= o[ax] < cmax[ax]):
                            tin, tout = 1.0, 0.0
                        continue
                    ta = (cmin[ax] - o[ax]) / u[ax]
                    tb = (cmax[ax] - o[ax]) / u[ax]
                    tin = max(tin, min(ta, tb))
                    tout = min(tout, max(ta, tb))
                if abs(tout - tin) < margin:
                    amb = True
                if tout - tin > 0:
                    cells.add((i, j, k))
    return cells, amb


def test_dda_brute_force_tiny_grid():
    """The band DDA enters exactly the cells the band segment meets (seeded
    random rays in a < 16^3 grid; rays with a near-grazing cell are skipped)."""
    rng = np.random.default_rng(7)
    p = oracle.make_params(V, TAU)
    checked = 0
    for _ in range(400):
        pose = _rand_pose(rng, 0.4)
        pt = rng.uniform(-0.6, 0.6, 3).astype(np.float32)
        if np.linalg.norm(pt) < 0.05:
            continue
        vis = oracle.point_visits(p, pt, pose)
        assert vis is not None
        x = pose[:3, :3] @ pt.astype(np.float64) + pose[:3, 3]
        cells, amb = _segment_cells_fp64(pose[:3, 3], x, TAU, V, 1e-5)
        if amb:
            continue
        got = [tuple(c) for c in vis.tolist()]
        assert len(set(got)) == len(got), "a voxel was entered twice"
        assert set(got) == cells
        # consecutive voxels are face neighbours
        assert (np.abs(np.diff(vis, axis=0)).sum(axis=1) == 1).all()
        checked += 1
    assert checked > 300


def test_pair_sdf_and_filter():
    """Kept pairs have d = (x - c) . u (to FP32 rounding) clamped to tau; the
    dropped visits are exactly those with d < -tau."""
    rng = np.random.default_rng(11)
    p = oracle.make_params(V, TAU)
    for _ in range(100):
        pose = _rand_pose(rng, 2.0)
        pt = rng.uniform(-4, 4, 3).astype(np.float32)
        vis = oracle.point_visits(p, pt, pose)
        x = pose[:3, :3] @ pt.astype(np.float64) + pose[:3, 3]
        u = (x - pose[:3, 3]) / np.linalg.norm(x - pose[:3, 3])
        dref = ((x[None, :] - (vis + 0.5) * V) * u[None, :]).sum(axis=1)
        ijk, _, d = oracle.scan_pairs(p, pt[None, :], pose)
        clear = np.abs(dref + TAU) > 1e-5
        kept = dref >= -TAU
        assert len(d) == kept.sum() or not clear.all()
        if clear.all():
            assert np.array_equal(ijk, vis[kept])
            np.testing.assert_allclose(d, np.minimum(dref[kept], TAU), atol=5e-6)
            assert (d <= np.float32(TAU)).all() and (d >= -np.float32(TAU)).all()


def test_invalid_points():
    p = oracle.make_params(V, TAU, min_range=1.0, max_range=10.0)
    o = np.eye(4)
    for bad in [[0.5, 0, 0], [11, 0, 0], [np.nan, 1, 1], [np.inf, 0, 0], [0, 0, 0]]:
        assert oracle.point_visits(p, bad, o) is None
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=3, min_range=1.0, max_range=10.0)
    assert m.integrate(np.zeros((0, 3)), o, np.zeros((0, 3))) == 0
    assert m.integrate([[0.5, 0, 0], [np.nan, 0, 0]], o, np.ones((2, 3))) == 0
    assert m.count() == 0


def test_fp32_vs_fp64_geometry_close():
    """The FP32 operation order stays within rounding of the FP64 geometry:
    almost all voxels agree and the shared voxels' D agree to ~1e-6."""
    w = synth.room_lidar(n_scans=2, n_beams=8, n_az=128)
    res = []
    for f64 in (False, True):
        m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=10, min_range=0.1,
                             max_range=100.0, fp64_geometry=f64)
        for s in w.scans:
            m.integrate(s["pts"], s["pose"], s["sem"])
        res.append(m.extract())
    a, b = res
    ka = {tuple(k) for k in a["ijk"].tolist()}
    kb = {tuple(k) for k in b["ijk"].tolist()}
    assert len(ka ^ kb) <= 1e-3 * len(ka)


# ----------------------------------------------------------------- fusion pins
def _groupby_pairs(params, scans):
    """Per-voxel observation lists from the oracle's pair generator."""
    obs = {}
    for si, s in enumerate(scans):
        ijk, pt, d = oracle.scan_pairs(params, s["pts"], s["pose"])
        for k in range(len(d)):
            obs.setdefault(tuple(ijk[k]), []).append((si, int(pt[k]), d[k]))
    return obs


def test_tsdf_counts_closed_forms():
    """W = number of observations, D = their mean (w~ = 1), one-hot counts =
    per-class observation counts (Theorem 1), sum c = W, posterior sums to 1."""
    w = synth.room_lidar(n_scans=3, n_beams=8, n_az=96)
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=10, min_range=0.1, max_range=100.0)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    e = m.extract()
    obs = _groupby_pairs(m.params, w.scans)
    assert len(obs) == len(e["W"])
    for k, key in enumerate(map(tuple, e["ijk"].tolist())):
        lst = obs[key]
        assert e["W"][k] == len(lst)
        assert e["D"][k] == pytest.approx(np.mean([x[2] for x in lst]), rel=1e-12, abs=1e-15)
        cnt = np.zeros(10)
        for si, j, _ in lst:
            cnt[int(np.argmax(w.scans[si]["sem"][j]))] += 1
        assert np.array_equal(e["sem"][k], cnt)
    assert np.array_equal(e["sem"].sum(axis=1), e["W"])
    post = m.extract(posterior=True)["sem"]
    np.testing.assert_allclose(post.sum(axis=1), 1.0, rtol=1e-14)


def test_posterior_single_class_and_alpha0():
    o = _pose_t(0.05, 0.05, 0.05)
    for a0 in (0.0, 1.0, 2.5):
        m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=5, alpha0=a0)
        for r in (1.02, 1.03, 1.04):
            m.integrate([[r, 0, 0]], o, _onehot_probs(np.array([3]), 5))
        e = m.extract(posterior=True)
        W = m.extract()["W"]
        for k in range(len(W)):
            exp = np.full(5, a0 / (5 * a0 + W[k]))
            exp[3] = (a0 + W[k]) / (5 * a0 + W[k])
            np.testing.assert_allclose(e["sem"][k], exp, rtol=1e-15)


def test_order_and_split_independence():
    """Theorems 1-2 hold for observation sets: scan order and any split of a
    scan into several calls give the same posterior (to FP64 rounding)."""
    w = synth.room_lidar(n_scans=3, n_beams=8, n_az=64)
    for mode, K, L in ((oracle.CLOSED_ONEHOT, 10, 0), (oracle.CLOSED_SOFT, 10, 0)):
        outs = []
        for order in ([0, 1, 2], [2, 0, 1], "split"):
            m = oracle.OracleMap(voxel_size=V, trunc=TAU, mode=mode, num_classes=K,
                                 min_range=0.1, max_range=100.0)
            if order == "split":
                for s in w.scans[::-1]:
                    h = s["pts"].shape[0] // 3
                    m.integrate(s["pts"][h:], s["pose"], s["sem"][h:])
                    m.integrate(s["pts"][:h], s["pose"], s["sem"][:h])
            else:
                for i in order:
                    m.integrate(w.scans[i]["pts"], w.scans[i]["pose"], w.scans[i]["sem"])
            outs.append(m.extract())
        for o in outs[1:]:
            assert np.array_equal(o["ijk"], outs[0]["ijk"])
            assert np.array_equal(o["W"], outs[0]["W"])
            np.testing.assert_allclose(o["D"], outs[0]["D"], rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(o["sem"], outs[0]["sem"], rtol=1e-12, atol=1e-13)


def _open_scans(n_scans=3, dim=6, seed=5):
    w = synth.indoor_rgbd(seed=seed, n_frames=40, width=24, height=18, dim=dim,
                          frames=list(range(n_scans)))
    return w


def test_open_set_theorem2_batch_form():
    """The oracle's one-observation recursion equals Theorem 2 applied once per
    scan to that scan's observation set (Eqs. norm_update_1-4), with lambda
    and nu tracked separately from zero priors; lambda = 2 nu = W holds."""
    w = _open_scans()
    m = oracle.OracleMap(voxel_size=0.05, trunc=0.15, mode=oracle.OPEN, embed_dim=6,
                         min_range=0.3, max_range=8.0)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    e = m.extract()
    state = {}
    for s in w.scans:
        ijk, pt, _ = oracle.scan_pairs(m.params, s["pts"], s["pose"])
        per = {}
        for k in range(len(pt)):
            per.setdefault(tuple(ijk[k]), []).append(s["sem"][pt[k]].astype(np.float64))
        for key, zs in per.items():
            Z = np.array(zs)
            n = Z.shape[0]
            zbar = Z.mean(axis=0)
            mm, lam, nu, beta = state.get(key, (np.zeros(6), 0.0, 0.0, np.zeros(6)))
            lam_t = lam + n
            m_t = (lam * mm + n * zbar) / lam_t
            nu_t = nu + n / 2.0
            beta_t = beta + 0.5 * ((Z - zbar) ** 2).sum(axis=0) + \
                (lam * n / lam_t) * (zbar - mm) ** 2 / 2.0
            state[key] = (m_t, lam_t, nu_t, beta_t)
    assert len(state) == len(e["W"])
    for k, key in enumerate(map(tuple, e["ijk"].tolist())):
        m_t, lam_t, nu_t, beta_t = state[key]
        assert lam_t == e["W"][k] and 2 * nu_t == e["W"][k]
        np.testing.assert_allclose(e["sem"][k], m_t, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(e["beta"][k], beta_t, rtol=1e-9, atol=1e-14)


def test_open_set_textbook_and_identical():
    """Zero priors: m = sample mean, beta = 1/2 sum of squared deviations;
    identical observations give m = z and beta = 0."""
    w = _open_scans(n_scans=2)
    m = oracle.OracleMap(voxel_size=0.05, trunc=0.15, mode=oracle.OPEN, embed_dim=6,
                         min_range=0.3, max_range=8.0)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    e = m.extract()
    per = {}
    for s in w.scans:
        ijk, pt, _ = oracle.scan_pairs(m.params, s["pts"], s["pose"])
        for k in range(len(pt)):
            per.setdefault(tuple(ijk[k]), []).append(s["sem"][pt[k]].astype(np.float64))
    for k, key in enumerate(map(tuple, e["ijk"].tolist())):
        Z = np.array(per[key])
        np.testing.assert_allclose(e["sem"][k], Z.mean(axis=0), rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(e["beta"][k], 0.5 * ((Z - Z.mean(0)) ** 2).sum(0),
                                   rtol=1e-9, atol=1e-14)
    z = np.array([0.3, -0.2, 0.5, 0.1, 0.0, 0.7], np.float32)
    m2 = oracle.OracleMap(voxel_size=0.05, trunc=0.15, mode=oracle.OPEN, embed_dim=6,
                          min_range=0.3, max_range=8.0)
    for s in w.scans:
        m2.integrate(s["pts"], s["pose"], np.tile(z, (s["pts"].shape[0], 1)))
    e2 = m2.extract()
    np.testing.assert_allclose(e2["sem"], np.tile(z.astype(np.float64), (len(e2["W"]), 1)),
                               rtol=1e-14)
    assert np.abs(e2["beta"]).max() < 1e-14


def test_extract_order():
    w = synth.room_lidar(n_scans=1, n_beams=8, n_az=64)
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=10, min_range=0.1, max_range=100.0)
    m.integrate(w.scans[0]["pts"], w.scans[0]["pose"], w.scans[0]["sem"])
    ijk = m.extract()["ijk"].astype(np.int64)
    b = np.floor_divide(ijk, 8)
    loc = ((ijk[:, 0] - 8 * b[:, 0]) * 8 + (ijk[:, 1] - 8 * b[:, 1])) * 8 + (ijk[:, 2] - 8 * b[:, 2])
    keys = list(zip(b[:, 0], b[:, 1], b[:, 2], loc))
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_query_brute_force():
    rng = np.random.default_rng(3)
    rows = rng.standard_normal((50, 16))
    rows[7] = 0.0
    q = synth.random_queries(4, 32, 16)
    label, prob, cos = oracle.query(rows, q, 0.05, 0.1)
    q64 = q.astype(np.float64)
    c = (rows @ q64.T) / np.maximum(
        np.linalg.norm(rows, axis=1, keepdims=True), 1e-300) / np.linalg.norm(q64, axis=1)[None]
    best = np.argmax(c, axis=1)
    e = np.exp((c - c.max(1, keepdims=True)) / 0.05)
    pb = e.max(1) / e.sum(1)
    for i in range(50):
        if i == 7:
            assert label[i] == -1 and prob[i] == 0
            continue
        assert prob[i] == pytest.approx(pb[i], rel=1e-12)
        assert label[i] == (best[i] if pb[i] >= 0.1 else -1)
        np.testing.assert_allclose(cos[i], c[i], rtol=1e-12, atol=1e-14)


# -------------------------------------------------------------- gradient pins
def _fd_map(params_kw, scans):
    m = oracle.OracleMap(**params_kw)
    for s in scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    return m


def test_backward_closed_soft_fd():
    """The oracle's adjoint matches central finite differences of its own
    FP64-geometry forward pass (pair sets held fixed by choice of h)."""
    rng = np.random.default_rng(12)
    w = synth.room_lidar(n_scans=2, n_beams=6, n_az=40, K=5, mode="soft")
    kw = dict(voxel_size=V, trunc=TAU, mode=oracle.CLOSED_SOFT, num_classes=5,
              min_range=0.1, max_range=100.0, alpha0=1.0)
    base = _fd_map(kw, w.scans)
    e = base.extract()
    nv = len(e["W"])
    a = rng.standard_normal(nv)
    B = rng.standard_normal((nv, 5))
    keys = e["ijk"]

    def loss(ext):
        assert np.array_equal(ext["ijk"], keys)
        c = ext["sem"]
        post = (1.0 + c) / (5.0 + c.sum(1, keepdims=True))
        return float((a * ext["D"] ** 2).sum() + (B * np.log(post)).sum())

    c = e["sem"]
    tot = 5.0 + c.sum(1, keepdims=True)
    gD = 2 * a * e["D"]
    gS = B / (1.0 + c) - B.sum(1, keepdims=True) / tot
    s0 = w.scans[0]
    gsem, gxyz = base.backward_scan(s0["pts"], s0["pose"], s0["sem"], gD, gS)
    kw64 = dict(kw, fp64_geometry=True)
    idx = rng.choice(np.flatnonzero(np.linalg.norm(s0["pts"], axis=1) > 0.1), 6, replace=False)
    for j in idx:
        for comp in range(3):
            h = 1e-4
            vals = []
            for sgn in (1, -1):
                sc = [dict(s) for s in w.scans]
                pts = s0["pts"].astype(np.float64).copy()
                pts[j, comp] += sgn * h
                sc[0]["pts"] = pts.astype(np.float32)
                # the perturbation is applied in float32; use the realised step
                vals.append((loss(_fd_map(kw64, sc).extract()), float(sc[0]["pts"][j, comp])))
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert gxyz[j, comp] == pytest.approx(fd, rel=2e-3, abs=2e-3)
        for k in range(5):
            h = 1e-3
            vals = []
            for sgn in (1, -1):
                sc = [dict(s) for s in w.scans]
                sem = s0["sem"].astype(np.float64).copy()
                sem[j, k] += sgn * h
                sc[0]["sem"] = sem.astype(np.float32)
                vals.append((loss(_fd_map(kw, sc).extract()), float(sc[0]["sem"][j, k])))
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert gsem[j, k] == pytest.approx(fd, rel=1e-3, abs=1e-5)


def test_backward_open_fd():
    rng = np.random.default_rng(13)
    w = _open_scans(n_scans=2, dim=4, seed=9)
    kw = dict(voxel_size=0.05, trunc=0.15, mode=oracle.OPEN, embed_dim=4,
              min_range=0.3, max_range=8.0)
    base = _fd_map(kw, w.scans)
    e = base.extract()
    nv = len(e["W"])
    A = rng.standard_normal((nv, 4))
    Bq = rng.standard_normal((nv, 4))

    def loss(ext):
        return float((A * ext["sem"] ** 2).sum() + (Bq * ext["beta"]).sum())

    gS = 2 * A * e["sem"]
    s1 = w.scans[1]
    gsem, _ = base.backward_scan(s1["pts"], s1["pose"], s1["sem"], np.zeros(nv), gS, Bq)
    idx = rng.choice(np.flatnonzero(np.linalg.norm(s1["pts"], axis=1) > 0.3), 5, replace=False)
    for j in idx:
        for k in range(4):
            h = 1e-3
            vals = []
            for sgn in (1, -1):
                sc = [dict(s) for s in w.scans]
                sem = s1["sem"].astype(np.float64).copy()
                sem[j, k] += sgn * h
                sc[1]["sem"] = sem.astype(np.float32)
                vals.append((loss(_fd_map(kw, sc).extract()), float(sc[1]["sem"][j, k])))
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert gsem[j, k] == pytest.approx(fd, rel=1e-3, abs=1e-6)


def test_dda_tie_breaks_to_lowest_axis():
    """On exact ties of the next crossing the DDA steps the lowest axis first
    (x, then y, then z): a (1,1,1) ray from a voxel centre crosses all three
    planes at the same t, so the visits cycle x, y, z."""
    p = oracle.make_params(V, TAU)
    o = _pose_t(0.05, 0.05, 0.05)
    for a in (0.7, 1.9):
        vis = oracle.point_visits(p, [a, a, a], o)
        steps = np.diff(vis, axis=0)
        axes = [int(np.flatnonzero(s)[0]) for s in steps]
        assert (np.abs(steps).sum(axis=1) == 1).all()
        assert len(axes) >= 4
        assert axes == [0, 1, 2] * (len(axes) // 3) + [0, 1, 2][:len(axes) % 3]


def test_uncertainty_closed_matches_scipy_dirichlet():
    """Closed-set uncertainty read-out: per-class variance of the Dirichlet
    posterior and entropy of its predictive, against scipy's Dirichlet and
    entropy routines (soft counts, alpha0 = 0.5)."""
    st = pytest.importorskip("scipy.stats")
    w = synth.room_lidar(seed=1, n_scans=2, K=10, mode="soft")
    m = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, mode=oracle.CLOSED_SOFT,
                         num_classes=10, min_range=w.min_range, max_range=w.max_range,
                         alpha0=0.5)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    ext = m.extract()
    unc = m.uncertainty()
    assert unc.shape == (len(ext["W"]), 11)
    rng = np.random.default_rng(0)
    for j in rng.choice(len(ext["W"]), 50, replace=False):
        alpha = 0.5 + ext["sem"][j]
        np.testing.assert_allclose(unc[j, :10], st.dirichlet(alpha).var(), rtol=1e-12)
        np.testing.assert_allclose(unc[j, 10], st.entropy(alpha / alpha.sum()), rtol=1e-12)


def test_uncertainty_open_matches_scipy_student_t():
    """Open-set uncertainty read-out: the variance of the Student-t predictive
    t_{2 nu}(m, beta (lambda + 1) / (lambda nu)) with lambda = 2 nu = W,
    against scipy's t distribution; infinite where 2 nu <= 2."""
    st = pytest.importorskip("scipy.stats")
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=48, height=36, dim=16, frames=[0, 1])
    m = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, mode=oracle.OPEN, embed_dim=16,
                         min_range=w.min_range, max_range=w.max_range)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    ext = m.extract()
    unc = m.uncertainty()
    W = ext["W"]
    assert (W <= 2).any() and (W > 2).any()
    assert np.all(np.isinf(unc[W <= 2]))
    for j in np.flatnonzero(W > 2)[:40]:
        lam, nu = W[j], W[j] / 2.0
        scale = np.sqrt(ext["beta"][j] * (lam + 1.0) / (lam * nu))
        ref = st.t(df=2.0 * nu, loc=ext["sem"][j], scale=scale).var()
        np.testing.assert_allclose(unc[j], ref, rtol=1e-12)


# ----------------------------------------------------------------- render
def _cam_forward_x(o):
    """world_from_camera: camera at o looking along +x (camera x -> world -y,
    camera y -> world -z)."""
    T = np.eye(4)
    T[:3, :3] = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    T[:3, 3] = o
    return T


def test_render_traversal_brute_force():
    """The render ray of a pixel enters exactly the cells its [near, far]
    segment meets (seeded poses and pixels; near-grazing cells skipped)."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(300):
        pose = _rand_pose(rng, 0.4)
        fx, fy, cx, cy = 60.0, 55.0, 32.0, 24.0
        px, py = int(rng.integers(0, 64)), int(rng.integers(0, 48))
        near, far = float(rng.uniform(0.0, 0.2)), float(rng.uniform(0.4, 0.9))
        vis = oracle.pixel_visits(V, pose, fx, fy, cx, cy, px, py, near, far)
        d = np.array([(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0])
        u = pose[:3, :3] @ (d / np.linalg.norm(d))
        o = pose[:3, 3]
        mid, half = 0.5 * (near + far), 0.5 * (far - near)
        cells, amb = _segment_cells_fp64(o, o + mid * u, half, V, 1e-5)
        if amb:
            continue
        got = [tuple(c) for c in vis.tolist()]
        assert len(set(got)) == len(got)
        assert set(got) == cells
        assert (np.abs(np.diff(vis, axis=0)).sum(axis=1) == 1).all()
        checked += 1
    assert checked > 200


def _plane_map(mode=oracle.CLOSED_ONEHOT, X0=2.0, dim=8, z=None):
    """A map of the plane x = X0 observed from the origin: a 60 x 60 fan of
    rays whose points lie on the plane (class 2 of 3, or embedding z)."""
    v, tau = 0.05, 0.15
    a = np.linspace(-0.4, 0.4, 60)
    A, B = np.meshgrid(a, a, indexing="ij")
    dirs = np.stack([np.ones_like(A), A, B], -1).reshape(-1, 3)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = (dirs * (X0 / dirs[:, 0])[:, None]).astype(np.float32)
    if mode == oracle.OPEN:
        m = oracle.OracleMap(voxel_size=v, trunc=tau, mode=mode, embed_dim=dim)
        sem = np.tile(z, (len(pts), 1)).astype(np.float32)
    else:
        m = oracle.OracleMap(voxel_size=v, trunc=tau, mode=mode, num_classes=3)
        sem = np.tile(np.array([0.1, 0.2, 0.7], np.float32), (len(pts), 1))
    m.integrate(pts, np.eye(4), sem)
    return m, v


def test_render_plane_depth_closed_form():
    """Rendering a plane x = X0 from the scan origin: every central pixel
    hits, the depth is the ray distance to the plane X0 / u_x, and the label
    is the plane's class. Depth error bound: a voxel is observed by scan rays
    up to its angular half-size (sqrt(3) v / 2) / r away from the render ray,
    over which the ray distance to the plane X0 / cos(theta) changes by
    (sqrt(3) v / 2) tan(theta) at incidence angle theta (plus rounding)."""
    X0 = 2.0
    m, v = _plane_map(X0=X0)
    W, H, f = 40, 30, 60.0
    out = m.render(_cam_forward_x(np.zeros(3)), f, f, W / 2, H / 2, W, H, 0.3, 6.0)
    d = np.stack(np.meshgrid((np.arange(W) + 0.5 - W / 2) / f, (np.arange(H) + 0.5 - H / 2) / f,
                             indexing="xy"), -1)
    ux = 1.0 / np.sqrt(1.0 + (d ** 2).sum(-1))  # world x component of the unit ray
    true = X0 / ux
    hit = np.isfinite(out["depth"])
    assert hit[5:-5, 5:-5].all()
    tan = np.sqrt(1.0 - ux ** 2) / ux
    bound = np.sqrt(3.0) / 2.0 * v * tan + 0.01 * v
    assert (np.abs(out["depth"] - true)[hit] <= bound[hit]).all()
    assert (out["label"][hit] == 2).all()
    assert (out["ijk"][hit][:, 0] * v <= X0 + v).all()


def test_render_miss_and_behind():
    """A camera looking away from the only surface sees nothing: depth +inf,
    label -1, indices INT32_MIN."""
    m, v = _plane_map()
    T = _cam_forward_x(np.zeros(3))
    T[:3, :3] = -T[:3, :3] @ np.diag([1.0, -1.0, 1.0])  # look along -x
    out = m.render(T, 50.0, 50.0, 16, 12, 32, 24, 0.1, 6.0)
    assert np.isinf(out["depth"]).all()
    assert (out["label"] == -1).all()
    assert (out["ijk"] == np.iinfo(np.int32).min).all()


def test_render_open_similarity():
    """Open set: the cosine of the hit voxel's mean with the query is 1 for
    the observed embedding itself and 0 for an orthogonal query."""
    z = np.zeros(8, np.float32)
    z[3] = 2.0
    m, v = _plane_map(mode=oracle.OPEN, z=z)
    T = _cam_forward_x(np.zeros(3))
    same = m.render(T, 50.0, 50.0, 16, 12, 32, 24, 0.3, 6.0, q=z)
    hit = np.isfinite(same["depth"])
    assert hit.sum() > 300
    np.testing.assert_allclose(same["sim"][hit], 1.0, atol=1e-12)
    q = np.zeros(8, np.float32)
    q[5] = 1.0
    orth = m.render(T, 50.0, 50.0, 16, 12, 32, 24, 0.3, 6.0, q=q)
    np.testing.assert_allclose(orth["sim"][hit], 0.0, atol=1e-12)
    assert (orth["label"] == -1).all()


def test_latest_label_mode_is_last_writer():
    """SLIM-VDB* (latest measurement wins): the label each voxel keeps is the
    argmax of the last observation in scan, then point, then ray order,
    replayed from the pair list; D and W are those of the Bayesian modes."""
    w = synth.room_lidar(seed=1, n_scans=3, K=10)
    kw = dict(voxel_size=w.voxel_size, trunc=w.trunc, num_classes=10, min_range=w.min_range,
              max_range=w.max_range)
    lat = oracle.OracleMap(mode=oracle.CLOSED_LATEST, **kw)
    hot = oracle.OracleMap(mode=oracle.CLOSED_ONEHOT, **kw)
    p = oracle.make_params(w.voxel_size, w.trunc, mode=oracle.CLOSED_LATEST, num_classes=10,
                           min_range=w.min_range, max_range=w.max_range)
    last = {}
    for s in w.scans:
        lat.integrate(s["pts"], s["pose"], s["sem"])
        hot.integrate(s["pts"], s["pose"], s["sem"])
        ijk, pt, _ = oracle.scan_pairs(p, s["pts"], s["pose"])
        lab = np.argmax(s["sem"], axis=1)
        for k, j in zip(map(tuple, ijk.tolist()), pt.tolist()):
            last[k] = lab[j]
    e, h = lat.extract(), hot.extract()
    assert np.array_equal(e["ijk"], h["ijk"])
    np.testing.assert_array_equal(e["W"], h["W"])
    np.testing.assert_allclose(e["D"], h["D"], rtol=0, atol=0)
    assert np.all(e["sem"].sum(1) == 1.0)
    got = np.argmax(e["sem"], axis=1)
    want = np.array([last[tuple(k)] for k in e["ijk"].tolist()])
    assert np.array_equal(got, want)
    # the ablation differs from the Bayesian counts wherever labels disagree
    assert (got != np.argmax(h["sem"], axis=1)).any()


def test_integrate_depth_backprojection():
    """RGB-D front end: integrating a z-depth image equals integrating the
    points back-projected in FP32 as ((u + 0.5 - cx) / fx * z, ...,  z) (numpy
    float32, same op order), bit for bit; invalid depths are skipped; the
    principal-point pixel back-projects onto the optical axis."""
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=64, height=48, dim=16, frames=[2])
    s = w.scans[0]
    H, W_ = 48, 64
    f = np.float32(525.0 * W_ / 640.0)
    cx, cy = np.float32(W_ / 2), np.float32(H / 2)
    depth = s["pts"][:, 2].reshape(H, W_).astype(np.float32).copy()
    depth[0, :5] = np.nan
    depth[1, :5] = -1.0
    u = np.arange(W_, dtype=np.float32)[None, :] + np.float32(0.5)
    v = np.arange(H, dtype=np.float32)[:, None] + np.float32(0.5)
    xu = ((u - cx) / f).astype(np.float32)
    yv = ((v - cy) / f).astype(np.float32)
    pts = np.stack([np.broadcast_to(xu, (H, W_)) * depth, np.broadcast_to(yv, (H, W_)) * depth,
                    depth], -1).reshape(-1, 3).astype(np.float32)
    pts[~(np.isfinite(depth) & (depth > 0)).reshape(-1)] = np.nan  # invalid pixels
    kw = dict(voxel_size=w.voxel_size, trunc=w.trunc, mode=oracle.OPEN, embed_dim=16,
              min_range=w.min_range, max_range=w.max_range)
    a, b = oracle.OracleMap(**kw), oracle.OracleMap(**kw)
    na = a.integrate_depth(depth, f, f, cx, cy, s["pose"], s["sem"])
    nb = b.integrate(pts, s["pose"], s["sem"])
    assert na == nb and na < H * W_ - 9
    ea, eb = a.extract(), b.extract()
    for k in ("ijk", "W", "D", "sem", "beta"):
        assert np.array_equal(ea[k], eb[k]), k
    # one valid pixel at the principal point: a ray along the optical axis
    one = np.zeros((2, 2), np.float32)
    one[1, 1] = 1.0
    c = oracle.OracleMap(voxel_size=0.1, trunc=0.3, mode=oracle.CLOSED_ONEHOT, num_classes=2,
                         min_range=0.1, max_range=10.0)
    c.integrate_depth(one, 1.0, 1.0, 1.5, 1.5, np.eye(4), np.full((4, 2), 0.5, np.float32))
    e = c.extract()
    assert len(e["W"]) > 0 and (e["ijk"][:, :2] == 0).all()
    np.testing.assert_allclose(e["D"], np.clip(1.0 - (e["ijk"][:, 2] + 0.5) * 0.1, -0.3, 0.3),
                               atol=1e-6)


# ------------------------------------------------------- weighting w~ != 1
def test_weighting_linear_axis_ray():
    """A ray along +x with the linear behind-surface weighting: each band
    voxel's d is x_0 - c (the axis-ray closed form); voxels in front of
    -eps keep weight 1, those behind carry (tau + d) / (tau - eps), falling
    to 0 at d = -tau, where the voxel stays out of the map."""
    eps = V
    o = _pose_t(0.05, 0.05, 0.05)
    for r in [1.3337, 2.71, 7.77]:
        m = oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=3, weighting=1,
                             weight_eps=eps)
        m.integrate([[r, 0, 0]], o, _onehot_probs(np.array([2]), 3))
        e = m.extract()
        x0 = 0.05 + r
        c = (e["ijk"][:, 0] + 0.5) * V
        d = np.minimum(x0 - c, TAU)
        w = np.where(d >= -eps, 1.0, (TAU + d) / (TAU - eps))
        np.testing.assert_allclose(e["W"], w, atol=1e-5)
        assert (e["W"] > 0).all() and (e["W"] <= 1).all()
        np.testing.assert_allclose(e["D"], d, atol=2e-6)  # one observation: D = d
        np.testing.assert_allclose(e["sem"][:, 2], e["W"], rtol=1e-15)
        # weights never increase with depth along the ray
        assert (np.diff(e["W"][np.argsort(c)]) <= 1e-12).all()


def test_weighting_keeps_front_voxels_and_sums():
    """Invariants against the w~ = 1 map of the same scans: a voxel all of
    whose observations lie in front of -eps is unchanged; every other voxel
    has a smaller W; one-hot and soft counts still sum to W."""
    w = synth.room_lidar(n_scans=3, n_beams=8, n_az=96)
    eps = 0.5 * V
    kw = dict(voxel_size=V, trunc=TAU, num_classes=10, min_range=0.1, max_range=100.0)
    maps = {}
    for mode in (oracle.CLOSED_ONEHOT, oracle.CLOSED_SOFT):
        for wt in (0, 1):
            m = oracle.OracleMap(mode=mode, weighting=wt, weight_eps=eps, **kw)
            for s in w.scans:
                m.integrate(s["pts"], s["pose"], s["sem"])
            maps[mode, wt] = m.extract()
    obs = _groupby_pairs(oracle.make_params(**kw), w.scans)
    for mode in (oracle.CLOSED_ONEHOT, oracle.CLOSED_SOFT):
        u, g = maps[mode, 0], maps[mode, 1]
        gi = {tuple(k): i for i, k in enumerate(g["ijk"].tolist())}
        front = 0
        for k, key in enumerate(map(tuple, u["ijk"].tolist())):
            dmin = min(x[2] for x in obs[key])
            if dmin >= -eps:
                front += 1
                i = gi[key]
                assert g["W"][i] == u["W"][k] and g["D"][i] == u["D"][k]
                assert np.array_equal(g["sem"][i], u["sem"][k])
            elif key in gi:
                assert g["W"][gi[key]] < u["W"][k]
        assert front > 0
        np.testing.assert_allclose(g["sem"].sum(axis=1), g["W"], rtol=1e-6)


def test_weighting_refused_for_open_set_and_adjoint():
    with pytest.raises(ValueError):
        oracle.OracleMap(voxel_size=V, trunc=TAU, mode=oracle.OPEN, embed_dim=8, weighting=1,
                         weight_eps=0.05)
    with pytest.raises(ValueError):
        oracle.OracleMap(voxel_size=V, trunc=TAU, num_classes=3, weighting=1, weight_eps=TAU)
    m = oracle.OracleMap(voxel_size=V, trunc=TAU, mode=oracle.CLOSED_SOFT, num_classes=3,
                         weighting=1, weight_eps=0.05)
    p = np.array([[1.0, 0.2, 0.1]], np.float32)
    s = np.array([[0.2, 0.3, 0.5]], np.float32)
    m.integrate(p, _pose_t(0, 0, 0), s)
    e = m.extract()
    with pytest.raises(RuntimeError):
        m.backward_scan(p, _pose_t(0, 0, 0), s, np.zeros(len(e["W"])), np.zeros((len(e["W"]), 3)))
