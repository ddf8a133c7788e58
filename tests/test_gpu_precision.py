"""Error of every output of the CUDA path against the FP64 oracle.

The parity tests compare with the oracle in parity mode (geometry in a fixed
FP32 operation order, fusion in FP64), which isolates the fusion arithmetic.
Here the reference is the oracle run entirely in FP64 (rays, DDA, pair SDFs
and fusion), so each number states what FP32 geometry, FP32 accumulation and,
for the open set, BF16 storage of m and beta cost together. The pose is
composed in FP64 on both sides. Each case prints one line per output
(``pytest -s``) and asserts the bound stated beside it.

Outputs (Sec. III-A to III-D): voxel key set, W, D, closed-set counts and the
Eq. dir_to_cat posterior, open-set NIG m and beta, and the query cosine."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _join(g, o):
    """Row indices of the voxels both maps hold, and the size of the
    symmetric difference of the key sets."""
    kg = {tuple(r): i for i, r in enumerate(g["ijk"])}
    ko = {tuple(r): i for i, r in enumerate(o["ijk"])}
    common = [k for k in kg if k in ko]
    ig = np.array([kg[k] for k in common], np.int64)
    io = np.array([ko[k] for k in common], np.int64)
    return ig, io, len(kg) + len(ko) - 2 * len(common)


def _report(case, what, value, bound):
    print(f"[precision] {case:<28} {what:<26} {value:.3e}  (bound {bound:.3e})")
    assert value <= bound, (case, what, value, bound)


def _geometry(case, g, o, max_keys, max_w):
    ig, io, sd = _join(g, o)
    n = len(o["W"])
    _report(case, "key set sym. diff / n", sd / n, max_keys)
    same = g["W"][ig].astype(np.float64) == o["W"][io]
    _report(case, "common voxels, W differs", 1.0 - same.mean(), max_w)
    return ig[same], io[same]


def _closed(case, w, mode, max_keys=0.0, max_w=0.0, **kw):
    alpha0, K = 1.0, w.num_classes
    g = to_np(gpu_map(w, mode=mode, **kw).extract(posterior=True))
    o = oracle_map(w, mode=mode, fp64=True).extract(posterior=True)
    ig, io = _geometry(case, g, o, max_keys, max_w)
    W = o["W"][io]
    # D: the pair SDFs carry FP32 geometry rounding (a few ulps of the
    # coordinates' magnitude) and are summed in FP32 (W ulps of tau)
    coord = float(np.abs(o["ijk"]).max() + 1) * w.voxel_size
    dD = np.abs(g["D"][ig] - o["D"][io])
    _report(case, "D abs err - W eps tau (m)", float((dD - W * EPS32 * w.trunc).max()),
            16 * EPS32 * coord)
    # the posterior returned by extract is (alpha0 + c) / (K alpha0 + W):
    # recover the counts to compare them too
    cg = g["sem"][ig] * (K * alpha0 + W)[:, None] - alpha0
    co = o["sem"][io] * (K * alpha0 + W)[:, None] - alpha0
    dc = np.abs(cg - co).max(axis=1)
    if mode == "onehot":
        _report(case, "count err (integers)", float(np.round(dc).max()), 0.0)
    else:
        # exact fixed-point sums (unit 2^-32) rounded once to FP32; the counts
        # recovered from the FP32 posterior carry its rounding times K + W
        _report(case, "soft count err / (K+W) eps", float((dc / ((K * alpha0 + W) * EPS32)).max()),
                8.0)
    dp = np.abs(g["sem"][ig] - o["sem"][io]).max()
    _report(case, "posterior abs err", float(dp), 1e-5)


def test_precision_room_onehot():
    _closed("room one-hot K=10", synth.room_lidar(n_scans=4, n_beams=16, n_az=256), "onehot")


def test_precision_room_soft():
    _closed("room soft K=20", synth.room_lidar(n_scans=4, n_beams=16, n_az=256, K=20,
                                               mode="soft"), "soft")


def test_precision_street_onehot():
    """Street coordinates reach ~80 m, where one FP32 ulp is ~8 um: a fraction
    of a percent of the band voxels lie on the other side of a DDA step or of
    the d >= -tau cut than in FP64."""
    _closed("street one-hot K=20", synth.street_lidar(n_scans=3, n_az=256), "onehot",
            max_keys=0.02, max_w=0.05)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_precision_open(storage):
    case = f"open l=64 {storage} storage"
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=64, height=48, dim=64,
                          frames=[0, 1, 2, 3])
    m = gpu_map(w, embed_storage=storage, voxel_capacity=200000)
    g = to_np(m.extract(index=True))
    o = oracle_map(w, fp64=True).extract()
    ig, io = _geometry(case, g, o, 0.0, 0.0)
    W = o["W"][io]
    coord = float(np.abs(o["ijk"]).max() + 1) * w.voxel_size
    dD = np.abs(g["D"][ig] - o["D"][io])
    _report(case, "D abs err - W eps tau (m)", float((dD - W * EPS32 * w.trunc).max()),
            16 * EPS32 * coord)
    n = len(w.scans)
    for k, ulp in (("sem", 2.0 ** -9), ("beta", 2.0 ** -8)):
        scale = np.abs(o[k]).max()
        err = float(np.abs(g[k][ig] - o[k][io]).max() / scale)
        # FP32: accumulation only; BF16: one storage rounding per scan (m) and
        # the next scan's beta update from the rounded m (beta)
        bound = 2e-5 if storage == "f32" else n * ulp
        _report(case, f"{'m' if k == 'sem' else 'beta'} err / max|ref|", err, bound)
    # query cosine: BF16 means (a BF16 copy of FP32 means) and BF16 queries
    # on tensor cores with FP32 accumulation, against FP64 means and queries
    qf = synth.random_queries(11, 64, 64)
    q = torch.from_numpy(qf).to(torch.bfloat16).cuda()
    _, _, sc = m.query(q, temperature=0.01, tp=0.1, scores=True)
    sc = sc.cpu().numpy()[g["index"][ig]]
    _, _, oc = oracle.query(o["sem"][io], qf, 0.01, 0.1)
    _report(case, "query cosine abs err", float(np.abs(sc - oc).max()), 1e-2)
