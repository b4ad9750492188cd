"""The multi-GPU path is replicas only (a solve does not shard): N ranks each
run their own solve and the bench reports the cells of all ranks over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 * (rank + 1)                      # rank 1 is the slower replica
    v, ms = bench.replica_rate(ms_local, cells=1000, steps=5, dist=dist, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, v, ms))


def test_two_replicas_report_the_slowest_rank_and_all_cells():
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
    for rank, v, ms in res:
        assert ms == 20.0                              # max over ranks
        assert v == pytest.approx(2 * 1000 * 5 / 20e-3 / 1e6)   # all ranks' cells


def test_single_process_rate():
    import bench
    v, ms = bench.replica_rate(4.0, cells=2048 * 2048, steps=10, dist=None)
    assert ms == 4.0 and v == pytest.approx(2048 * 2048 * 10 / 4e-3 / 1e6)
