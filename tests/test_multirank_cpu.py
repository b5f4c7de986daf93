"""The multi-rank (N > 1) logic of bench.py on CPU ranks over gloo, world size 2.

Under weak scaling every rank convolves its own maps (no collective on the data
path); only the step time is reduced, with MAX, and the aggregate rate is the
units of all ranks over that time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from inputs import white_noise_maps
    dist.init_process_group("gloo", rank=rank, world_size=world)
    maps = white_noise_maps(4, 2, 5)
    mine = bench.shard_maps(maps, rank, world)
    step_s = 0.010 * (rank + 1)                      # rank 1 is the slower one
    t = bench.max_over_ranks(step_s, world, "cpu")
    rate = bench.aggregate_rate(1000.0, world, t)
    out[rank] = (float(mine.sum()), float(mine[0, 0]), t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_logic_world_size_2():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    (s0, first0, t0, r0), (s1, first1, t1, r1) = out[0], out[1]
    assert t0 == pytest.approx(0.020) and t1 == pytest.approx(0.020)        # MAX over ranks
    assert r0 == pytest.approx(1000.0 * 2 / 0.020) and r0 == r1
    assert s0 == pytest.approx(s1, rel=1e-6)        # same data, shifted: the sums agree
    assert first0 != first1                          # but each rank has its own maps
