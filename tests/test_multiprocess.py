"""The N > 1 path of bench.py on the CPU: replicas under torch.distributed
(gloo, world size 2), barrier, slowest-rank time, whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist()
    assert (ws, r, local) == (world, rank, rank)
    dist.barrier()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)           # rank 1 is slower
    val = bench.job_throughput(1e12, ms, ws)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, val in res:
        assert ms == 15.0                         # the max over ranks
        assert val == pytest.approx(2 * 1e12 / 0.015 / 1e12)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_throughput(2e12, 1000.0, 1) == pytest.approx(2.0)
