"""Shared helpers for the GPU parity tests: run the CUDA path and the oracle
on the same seeded inputs and compare them element by element."""
import os

import numpy as np

import oracle

# parity tolerance for FP32 fields (SDF, posteriors): relative, absolute
RTOL, ATOL = 1e-5, 1e-6


def oracle_map(w, mode=None, fp64=False, **kw):
    mode = w.mode if mode is None else mode
    mcode = {"onehot": oracle.CLOSED_ONEHOT, "soft": oracle.CLOSED_SOFT, "open": oracle.OPEN,
             "latest": oracle.CLOSED_LATEST}[mode]
    m = oracle.OracleMap(voxel_size=w.voxel_size, trunc=w.trunc, mode=mcode,
                         num_classes=w.num_classes, embed_dim=w.embed_dim,
                         min_range=w.min_range, max_range=w.max_range,
                         body_from_sensor=w.body_from_sensor, fp64_geometry=fp64, **kw)
    for s in w.scans:
        m.integrate(s["pts"], s["pose"], s["sem"])
    return m


def gpu_map(w, mode=None, scans=None, **kw):
    import torch
    from paper_2512_12945_gb300 import slim
    mode = w.mode if mode is None else mode
    args = dict(voxel_size=w.voxel_size, trunc=w.trunc, mode=mode, num_classes=max(w.num_classes, 1),
                embed_dim=w.embed_dim if w.embed_dim else 64, min_range=w.min_range,
                max_range=w.max_range, body_from_sensor=w.body_from_sensor,
                max_points=max(s["pts"].shape[0] for s in w.scans))
    if mode == "open":
        args["image_width"] = getattr(w, "image_width", 0)
    args.update(kw)
    m = slim.Map(**args)
    for s in (w.scans if scans is None else scans):
        m.integrate(torch.from_numpy(s["pts"]).cuda(), s["pose"], torch.from_numpy(s["sem"]).cuda())
    m.sync()
    return m


def to_np(ext):
    return {k: v.cpu().numpy() for k, v in ext.items()}


# Worst error / tolerance ratio of every assert_close check, per (test, field);
# printed at the end of the session (conftest.py) so the margin of each
# parity check is visible, not only its pass or fail.
MARGINS = {}


def assert_close(got, ref, rtol=RTOL, atol=ATOL, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    tol = atol + rtol * np.abs(ref)
    if err.size:
        key = (os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], what)
        MARGINS[key] = max(MARGINS.get(key, 0.0), float((err / tol).max()))
    bad = err > tol
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} outside rtol={rtol} "
                           f"atol={atol}; worst {err.max():.3g}")


def compare_closed(g, o, mode, rtol=RTOL, atol=ATOL):
    """g: GPU extract (numpy), o: oracle extract."""
    assert g["ijk"].shape == o["ijk"].shape, (g["ijk"].shape, o["ijk"].shape)
    assert np.array_equal(g["ijk"], o["ijk"]), "voxel key sets differ"
    assert np.array_equal(g["W"].astype(np.float64), o["W"]), "weights differ"
    if mode == "onehot":
        assert np.array_equal(g["sem"].astype(np.float64), o["sem"]), "class counts differ"
    else:
        assert_close(g["sem"], o["sem"], rtol, atol, "soft counts")
    assert_close(g["D"], o["D"], rtol, atol, "D")
