"""The N > 1 path of bench.py runs independent replicas (the Newton step does
not shard): the job's time is the maximum over ranks and the value is the
total work over that time.  Checked with two gloo ranks on the CPU."""

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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [1.0 + rank, 10.0 - rank, 0.5 * (rank + 1)]   # rank 1 is slower on the first and last entries
    t = bench.max_over_ranks(local, dist)
    v = bench.replica_throughput(world, 100000, 20, t[0])
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (t, v)


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        t, v = res[r]
        assert t == [2.0, 10.0, 1.0]
        assert v == pytest.approx(2 * 100000 * 20 / 2.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None) == [1.5, 2.5]
    assert bench.replica_throughput(1, 10, 3, 2.0) == 15.0
