"""The multi-replica path of bench.py on CPU: two gloo ranks with different
local times agree on the slowest rank's time, and the whole-job throughput
counts both ranks' work over it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.replica_throughput(10.0 + 5.0 * rank, 1000, 30)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 * 30 / 15e-3)


def test_single_process_is_its_own_time():
    import bench
    ms, value = bench.replica_throughput(8.0, 500, 4)
    assert ms == 8.0 and value == pytest.approx(500 * 4 / 8e-3)
