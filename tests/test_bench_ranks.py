"""The multi-rank host logic of bench.py (one rank per GPU, independent
replicas): the job's time is the slowest rank's, and the job's throughput
counts every rank's voxels.  Two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 40.0][rank]
    got = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    dist.barrier()
    out[rank] = (got, bench.job_throughput(world, 1000, 10, got / 1e3))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 40.0
    # 2 ranks x 1000 voxels x 10 iterations in 40 ms
    assert out[0][1] == pytest.approx(2 * 1000 * 10 / 0.040 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.job_throughput(1, 10**9, 10, 2.0) == pytest.approx(5.0)
