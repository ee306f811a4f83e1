"""The multi-rank logic of bench.py (weak scaling: every rank runs its own independent
gradient; the timed region is bracketed by barriers and the slowest rank's time is
used) on two CPU ranks with the gloo backend."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    t = 10.0 + rank                      # the slower rank decides the time
    out[rank] = bench.reduce_max(t, w, torch.device("cpu"))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_ranks_take_the_max_time():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
