"""The multi-GPU form is replicas (one independent map per rank, no
collective on the data path): the benchmark's timing takes the slowest
rank's time over all ranks and counts every rank's points. Checked here with
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = 10.0 + 5.0 * rank  # the ranks finish at different times
    mx = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.replica_rate(ws, 1000, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, rate))


def test_two_replicas_max_time_and_total_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, rate in res:
        assert mx == 15.0  # the slowest rank
        assert rate == pytest.approx(2 * 1000 / 0.015)  # both ranks' units


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    sys_argv = sys.argv
    sys.argv = ["bench.py", "--impl", "reference"]
    try:
        assert bench.run_reference(bench.parse()) == 0
    finally:
        sys.argv = sys_argv
