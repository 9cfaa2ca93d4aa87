"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

Independent problems shard across GPUs with no collective on the data path;
the only cross-rank step is the max of the per-rank step times, and the job's
value counts every rank's voxels (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 10.0 - rank]           # rank 1 is slower on the first entry
        got = bench.max_over_ranks(mine)
        q.put((rank, got, bench.job_value(1000, world, got[0])))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [2.0, 10.0]
        assert value == pytest.approx(2 * 1000 / 2e-3)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_value(10, 1, 1.0) == pytest.approx(1e4)
