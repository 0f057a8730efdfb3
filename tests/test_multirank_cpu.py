"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the
drag step is cell local, so ranks share nothing but the timing reduction."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [100.0 + 50.0 * rank, 7.0 - rank, 3.0 * (rank + 1)]
    got = bench.max_over_ranks(local, world)
    rate = bench.whole_job_rate(1000, world, got[0])
    dist.barrier()
    dist.destroy_process_group()
    out_q.put((rank, got, rate))


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
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
    for rank, got, rate in res:
        assert got == [150.0, 7.0, 6.0]             # every rank sees the slowest rank's times
        assert rate == pytest.approx(2 * 1000 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)
