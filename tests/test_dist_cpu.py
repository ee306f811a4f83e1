"""The multi-rank logic on two CPU ranks with the gloo backend: bench.py's timing (the
timed region is bracketed by barriers and the slowest rank's time is used) and the
multi-shot gradient and GN-HVP (one shot per rank at the same wave speed, summed by one
all-reduce), which must equal the single-process sum of the per-shot oracle results."""
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


def _shot_problem(rank, world):
    import numpy as np
    from oracle import wave as W
    from paper_2304_04781_gb300 import inputs
    shape, nt = (16, 16, 16), 40
    src = inputs.source_grid(16, 16, 16, world)[rank]
    prob = W.Problem(shape=shape, h=10.0, nt=nt, rec=inputs.receiver_grid(16, 16, 16), src=src)
    c = inputs.velocity_model(shape, 10.0, seed=5)
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c))
    dc = inputs.direction(shape, 10.0, seed=12)
    return prob, c, d_obs, dc


def _shot_worker(rank, world, port, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import wave as W
    from paper_2304_04781_gb300 import multishot
    prob, c, d_obs, dc = _shot_problem(rank, world)

    def shot():
        J, g, _ = W.gradient(prob, c, d_obs)
        return J, torch.from_numpy(g)

    def shot_hv():
        _, states = W.forward_states(prob, c)
        return torch.from_numpy(W.hessvec_gn(prob, c, dc, lambda n: states[n][0]))

    J, g = multishot.multishot_gradient(shot)
    h = multishot.multishot_hessvec(shot_hv)
    out[rank] = (J, g.numpy(), h.numpy())
    dist.destroy_process_group()


def test_two_shots_sum_to_the_single_process_sum():
    import numpy as np
    from oracle import wave as W
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_shot_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    Js, gs, hs = [], [], []
    for r in range(world):
        prob, c, d_obs, dc = _shot_problem(r, world)
        J, g, _ = W.gradient(prob, c, d_obs)
        _, states = W.forward_states(prob, c)
        Js.append(J)
        gs.append(g)
        hs.append(W.hessvec_gn(prob, c, dc, lambda n: states[n][0]))
    # the shots differ, so the sum is not a multiple of one of them
    assert np.linalg.norm(gs[0] - gs[1]) > 0.1 * np.linalg.norm(gs[0])
    for r in range(world):
        J, g, h = out[r]
        assert J == pytest.approx(sum(Js), rel=1e-12)
        np.testing.assert_allclose(g, gs[0] + gs[1], rtol=0, atol=1e-12 * np.abs(gs[0] + gs[1]).max())
        np.testing.assert_allclose(h, hs[0] + hs[1], rtol=0, atol=1e-12 * np.abs(hs[0] + hs[1]).max())


def test_one_shot_is_the_centre_source():
    from paper_2304_04781_gb300 import inputs
    assert inputs.source_grid(256, 256, 256, 1) == [(128, 128, 128)]
    assert len(set(inputs.source_grid(64, 64, 64, 8))) == 8
