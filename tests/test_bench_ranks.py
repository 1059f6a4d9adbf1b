"""The multi-rank aggregation of bench.py (replicas, one per GPU) on CPU ranks
over gloo: whole-job value = all ranks' units / max over ranks of the timed
region, and the barrier does not deadlock."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    my = [2.0, 5.0][rank]
    value, tmax = bench.whole_job_value(1000, 4, my, world)
    out[rank] = (value, tmax)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax = out[r]
        assert tmax == 5.0
        assert value == pytest.approx(2 * 1000 * 4 / 5.0)


def test_single_rank_value():
    import bench
    v, t = bench.whole_job_value(10, 3, 2.0, 1)
    assert t == 2.0 and v == pytest.approx(15.0)
