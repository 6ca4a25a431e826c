"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank
simulates its own environment shard; the only collective is the max of the
per-rank times, and the whole-job rate counts every rank's env-steps over
the slowest rank's time."""
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
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.barrier_max(10.0 + 5.0 * rank, world)
    q.put((rank, t, bench.shard_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]  # every rank sees the slowest time
    assert res[0][2] != res[1][2]  # distinct environment shards


def test_aggregate_rate():
    import bench
    # 2 ranks x 65536 envs x 1000 steps x 5 rollouts in 1 s of the slowest rank
    assert bench.aggregate_rate(2, 65536, 1000, 5, 1000.0) == pytest.approx(2 * 65536 * 1000 * 5)
