"""The bench's multi-rank logic on CPU with gloo, world size 2: the timing is
the max over ranks, whole-job throughput counts every rank's units, and every
rank gets its own data shard."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(1.0 + rank * 2.5)           # rank times 1.0 s and 3.5 s
    v = bench.weak_scaling_value(1000, world, t)
    seeds = [bench.shard_seed(n, rank) for n in bench.SWEEP_CODES]
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v, seeds))


def test_two_rank_reduction_and_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, seeds in res:
        assert t == pytest.approx(3.5)                 # max over ranks
        assert v == pytest.approx(1000 * 2 / 3.5)      # all ranks' units over the slowest time
    assert set(res[0][3]).isdisjoint(res[1][3])        # distinct data shards


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(2.0) == 2.0
    assert bench.weak_scaling_value(10, 1, 2.0) == 5.0
