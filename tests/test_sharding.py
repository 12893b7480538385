"""Frequency sharding across ranks: independent problems (Sec. III.B sweeps the
frequency), no data-path collective.  Two gloo ranks on CPU check that the bench's batch
assignment covers every frequency exactly once per round of steps, with the
seed convention 1000 + frequency index, and that the max-over-ranks timing
reduction works."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, F, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    om = W.log_omegas(64)
    got = []
    for s in range(steps):
        shifts, seeds, idx = bench.batch_for(s, rank, world, F, om, 1000)
        assert np.allclose(shifts, 1j * om[idx])
        assert seeds == [1000 + i for i in idx]
        got.extend(idx)
    t = bench.max_over_ranks(dist, float(rank + 1), torch.device("cpu"))
    out[rank] = (got, t)
    dist.destroy_process_group()


@pytest.mark.parametrize("F,steps", [(8, 4), (16, 2)])
def test_two_rank_frequency_shards(F, steps):
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), F, steps, out), nprocs=world,
                       join=True, start_method="spawn")
    a, ta = out[0]
    b, tb = out[1]
    assert ta == tb == 2.0                      # max over ranks
    assert not set(a) & set(b)                  # disjoint shards
    assert sorted(a + b) == list(range(64))     # every frequency once
