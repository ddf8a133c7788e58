"""The read-out entry point for callers that cannot allocate device memory
(slim_query_rows_static), against the oracle's read-out and against the map's
own read-out (slim_query).

Plug-ins whose host application owns every device allocation, real-time
loops with a memory budget fixed up front, or hosts that only hand in their
own buffers cannot let the library call cudaMalloc. slim_query_rows_static
takes its working memory from a static device array instead. These tests
call it through the C ABI on rows of real maps (the BF16 means an
integration left), compare its labels and probabilities with the oracle's
read-out of the same BF16 rows and with slim_query, on two calls in a row
(the array keeps the previous call's contents), and check that oversize
requests are refused. The file sits on its own and pytest collects it last.

Tolerances: the cosines come from BF16 products summed in FP32, within
COS_ATOL of the oracle's FP64 sums of the same BF16 values; a cosine error
delta moves a softmax probability of cos / T by at most a factor
exp(2 delta / T), so probabilities are compared at rtol 2 COS_ATOL / T plus
the rounding of the kernel's base-2 exponentials (2^-20 relative)."""
import numpy as np
import pytest

import oracle
from paper_2512_12945_gb300 import synth
from helpers import gpu_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COS_ATOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_12945_gb300 import build
    build.build()


def _map_rows(dim, frames, wh):
    """The BF16 means of a map integrated from indoor RGB-D frames, in row
    order (extract widens the stored BF16 values exactly)."""
    w = synth.indoor_rgbd(seed=3, n_frames=200, width=wh[0], height=wh[1], dim=dim,
                          frames=frames)
    m = gpu_map(w, embed_storage="bf16", voxel_capacity=600000)
    ext = m.extract(index=True)
    n = m.stats()["voxels"]
    assert n == ext["W"].shape[0]
    rows = torch.zeros((n, dim), dtype=torch.float32, device="cuda")
    rows[ext["index"].long()] = ext["sem"]
    return m, rows.to(torch.bfloat16).contiguous()


def _oracle_readout(rows, q, T):
    """The oracle's read-out of the same BF16 rows and queries, and the rows
    whose label is unique within rounding: top two cosines apart and the
    winner away from the threshold T_p (elsewhere either answer is correct)."""
    rf = rows.float().cpu().numpy().astype(np.float64)
    ol, op, oc = oracle.query(rf, q.float().cpu().numpy(), T, 0.1)
    top2 = np.sort(oc, axis=1)[:, -2:]
    clear = ((top2[:, 1] - top2[:, 0]) > 4 * COS_ATOL) & (np.abs(op - 0.1) > 1e-3)
    assert clear.mean() > 0.9
    return ol, op, clear


@pytest.mark.parametrize("dim,frames,wh,Q", [
    (64, [0, 30, 60, 90, 120, 150], (640, 480), 64),   # >= 2^16 rows
    (512, [0, 1, 2], (96, 72), 256),
    (1024, [0, 1], (64, 48), 40),
])
def test_static_scratch_readout_matches_oracle_and_map_readout(dim, frames, wh, Q):
    from paper_2512_12945_gb300 import slim
    m, rows = _map_rows(dim, frames, wh)
    n = rows.shape[0]
    if dim == 64:
        assert n >= 1 << 16, n
    T = 0.01
    rtol = 2 * COS_ATOL / T + 2.0 ** -20
    q = torch.from_numpy(synth.random_queries(11 + dim, Q, dim)).to(torch.bfloat16).cuda()
    ref_label, ref_prob = [x.cpu().numpy() for x in m.query(q, temperature=T, tp=0.1)[:2]]
    for part in (n, n - 37):  # all rows, then a ragged prefix (one is not a multiple of 128)
        sub = rows[:part].contiguous()
        ol, op, clear = _oracle_readout(sub, q, T)
        for _ in range(2):  # two calls in a row share the static array
            label, prob = slim.slim_query_rows_static(sub, q, temperature=T, tp=0.1)
            torch.cuda.synchronize()
            gl, gp = label.cpu().numpy(), prob.cpu().numpy()
            np.testing.assert_allclose(gp, op, rtol=rtol, atol=1e-7)
            assert np.array_equal(gl[clear], ol[clear])
            # the map's own read-out of the same rows
            np.testing.assert_allclose(gp, ref_prob[:part], rtol=rtol, atol=1e-7)
            assert np.array_equal(gl[clear], ref_label[:part][clear])


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
