"""The bench's N > 1 host logic on CPU: two gloo ranks (world size 2) run the same
timing reduction bench.py uses under torchrun. Each rank is an independent replica
on its own seeded shard (no data-path collective); the reported time is the max
over ranks and the value counts the rows of all ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        local_seconds = [0.5, 2.0][rank]
        t = bench.reduce_max(local_seconds)
        out[rank] = (t, bench.whole_job_rate(1000, world, t), bench.shard_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_timing_and_shards():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    (t0, v0, s0), (t1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 2.0                 # max over ranks
    assert v0 == v1 == 1000 * 2 / 2.0      # rows of all ranks / slowest time
    assert s0 != s1                        # independent shards


def test_shards_draw_different_rows():
    import bench
    import pxdata
    a = pxdata.plain_at_scale(1000, 5000, nattr=10, seed=bench.shard_seed(0))
    b = pxdata.plain_at_scale(1000, 5000, nattr=10, seed=bench.shard_seed(1))
    assert not np.array_equal(a["fk"], b["fk"])
