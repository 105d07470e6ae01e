"""The N > 1 bench logic on CPU ranks (gloo, world size 2): one replica per rank,
barriers, the maximum of the per-rank times, and the whole-job rate = all units
processed / slowest rank's time.  No GPU is used."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(world)
    times = bench.reduce_max(10.0 + 5.0 * rank, world)   # rank 1 is the slow one
    rate, t = bench.aggregate(times, [1000] * world)
    out[rank] = (times, rate, t)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation_on_gloo():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    for r in range(2):
        times, rate, t = out[r]
        assert times == [10.0, 15.0]
        assert t == 15.0
        assert rate == pytest.approx(2000 / 15e-3)


def test_aggregate_single_rank():
    import bench
    rate, t = bench.aggregate([4.0], [400])
    assert t == 4.0 and rate == pytest.approx(1e5)
