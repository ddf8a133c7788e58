"""The read-out entry point for callers that cannot allocate device memory
(slim_query_rows_static) against the map's own read-out (slim_query).

Plug-ins whose host application owns every device allocation, real-time
loops with a memory budget fixed up front, or hosts that only hand in their
own buffers cannot let the library call cudaMalloc. slim_query_rows_static
takes its working memory from a static device array instead; this test
checks, through the C ABI, that it gives the same labels and probabilities as
slim_query on the same rows, on two calls in a row (the array keeps the
previous call's contents). It sits in a file of its own that pytest collects
last."""
import numpy as np
import pytest

from paper_2512_12945_gb300 import synth
from helpers import gpu_map, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def test_static_scratch_readout_matches_map_readout():
    from paper_2512_12945_gb300 import slim
    w = synth.indoor_rgbd(seed=3, n_frames=40, width=64, height=48, dim=128,
                          frames=[0, 1, 2])
    m = gpu_map(w, embed_storage="bf16", voxel_capacity=400000)
    ext = m.extract(index=True)
    n = m.stats()["voxels"]
    assert n == ext["W"].shape[0] and n > 3 * 128
    # the map's stored means as BF16 rows in row order (exact: extract widens
    # the stored BF16 values to float32)
    rows = torch.zeros((n, 128), dtype=torch.float32, device="cuda")
    rows[ext["index"].long()] = ext["sem"]
    rows = rows.to(torch.bfloat16).contiguous()
    for T, seed, Q in ((0.01, 11, 256), (0.05, 12, 40)):
        q = torch.from_numpy(synth.random_queries(seed, Q, 128)).to(torch.bfloat16).cuda()
        ref_label, ref_prob, ref_sc = m.query(q, temperature=T, tp=0.1, scores=True)
        sc = ref_sc.cpu().numpy()
        top2 = np.sort(sc, axis=1)[:, -2:]
        clear = ((top2[:, 1] - top2[:, 0]) > 1e-4) & (np.abs(ref_prob.cpu().numpy() - 0.1) > 1e-3)
        for _ in range(2):  # two calls in a row share the static scratch
            label, prob = slim.slim_query_rows_static(rows, q, temperature=T, tp=0.1)
            torch.cuda.synchronize()
            np.testing.assert_allclose(prob.cpu().numpy(), ref_prob.cpu().numpy(), rtol=2e-3,
                                       atol=1e-6)
            gl, rl = label.cpu().numpy(), ref_label.cpu().numpy()
            assert clear.mean() > 0.9
            assert np.array_equal(gl[clear], rl[clear])


def test_static_scratch_rejects_oversize():
    from paper_2512_12945_gb300 import slim
    rows = torch.zeros((8, 64), dtype=torch.bfloat16, device="cuda")
    q = torch.zeros((300, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(slim.SlimError) as e:
        slim.slim_query_rows_static(rows, q)
    assert e.value.status == 1
    L = slim.lib()
    import ctypes
    rc = L.slim_query_rows_static(ctypes.c_void_p(rows.data_ptr()), (1 << 20) + 1, 64,
                                  ctypes.c_void_p(q.data_ptr()), 4, 0.01, 0.1, None, None, None)
    assert rc == 1 and b"2^20" in L.slim_last_error()
