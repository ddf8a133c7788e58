"""Open-set query (tcgen05 BF16 GEMM + fused cosine / softmax / argmax /
threshold) against the oracle's read-out on the same map state: the oracle is
given the map's stored means (as stored, BF16 or FP32) and the BF16-rounded
queries, so the comparison isolates the tensor-core path (FP32 accumulation).
A second check states the error of the whole BF16 path against the FP64
oracle map."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import gpu_map, oracle_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _bf16_round(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16)


def _run(storage, dim, Q, frames=3, wh=(64, 48), T=0.01, tp=0.1):
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=wh[0], height=wh[1], dim=dim,
                          frames=list(range(frames)))
    m = gpu_map(w, embed_storage=storage, voxel_capacity=400000)
    ext = to_np(m.extract(index=True))
    q = _bf16_round(synth.random_queries(11, Q, dim)).cuda()
    label, prob, sc = m.query(q, temperature=T, tp=tp, scores=True)
    label, prob, sc = label.cpu().numpy(), prob.cpu().numpy(), sc.cpu().numpy()
    rows = m.stats()["voxels"]
    assert rows == len(ext["W"])
    # the map state as stored, in row order
    mrow = np.zeros((rows, dim))
    mrow[ext["index"]] = ext["sem"]
    if storage == "f32":  # the tensor cores read a BF16 copy of FP32-stored means
        mrow = _bf16_round(mrow).float().numpy().astype(np.float64)
    qf = q.float().cpu().numpy()
    ol, op, oc = oracle.query(mrow, qf, T, tp)
    return w, ext, (label, prob, sc), (ol, op, oc), q, m


@pytest.mark.parametrize("storage,dim,Q", [("bf16", 64, 256), ("f32", 64, 37),
                                           ("bf16", 512, 256), ("f32", 512, 16),
                                           ("bf16", 128, 200)])
def test_query_matches_oracle_readout(storage, dim, Q):
    _, ext, (gl, gp, gs), (ol, op, oc), _, _ = _run(storage, dim, Q)
    assert gs.shape == oc.shape
    np.testing.assert_allclose(gs, oc, atol=2e-5, rtol=0)
    # a cosine error delta moves the logit cos / T by delta / T and a softmax
    # probability by a factor of at most exp(2 delta / T); the kernel's
    # base-2 exponentials add 2^-20 relative
    delta = float(np.abs(gs - oc).max())
    np.testing.assert_allclose(gp, op, rtol=2 * delta / 0.01 + 2.0 ** -20, atol=1e-7)
    top2 = np.sort(oc, axis=1)[:, -2:] if Q > 1 else np.zeros((len(oc), 2))
    clear = (top2[:, 1] - top2[:, 0]) > 1e-4
    clear &= np.abs(op - 0.1) > 1e-3  # away from the threshold
    assert clear.mean() > 0.9
    assert np.array_equal(gl[clear], ol[clear])
    assert len(gl) > 3 * 128  # several tiles (plus a ragged tail)


def test_query_bf16_error_vs_fp64_oracle():
    """Whole BF16 path (BF16-stored means, BF16 queries) against the FP64
    oracle map and FP32 queries: cosine error stays within 1e-2."""
    w, ext, (gl, gp, gs), _, q, _ = _run("bf16", 64, 64)
    o = oracle_map(w).extract()
    assert np.array_equal(ext["ijk"], o["ijk"])
    qf = synth.random_queries(11, 64, 64)
    _, _, oc = oracle.query(o["sem"], qf, 0.01, 0.1)
    gs_by_voxel = gs[ext["index"]]
    err = np.abs(gs_by_voxel - oc)
    assert err.max() < 1e-2, err.max()


def test_query_rejects_bad_args():
    from paper_2512_12945_gb300 import slim
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=32, height=24, dim=64, frames=[0])
    m = gpu_map(w, voxel_capacity=100000)
    q = _bf16_round(synth.random_queries(1, 300, 64)).cuda()
    with pytest.raises(slim.SlimError):
        m.query(q)
    with pytest.raises(slim.SlimError):
        m.query(q[:4], temperature=0.0)
