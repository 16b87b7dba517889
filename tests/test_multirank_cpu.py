"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2).

Each rank traces its own seeds (weak scaling) and the only cross-rank traffic
is the timing barrier and the reduction of (slowest time, total steps); the
ranks here run the oracle on their own seed streams in place of the GPU path.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2606_02627_gb300 import inputs
    g = inputs.cube_grid(17)
    F = inputs.rotation_field(g)
    seeds = inputs.uniform_seeds(g, 64, bench.rank_seed(1, rank))
    dt = 0.25 / oracle.max_speed(F, g.spacing)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 40)
    steps = int(L.steps().sum())
    ms = 10.0 + rank                          # a stand-in timing: rank 1 is slower
    dist.barrier()
    ms_all, steps_all = bench.reduce_over_ranks(ms, steps, dist, "cpu")
    out[rank] = (ms_all, steps_all, steps, seeds[0].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_reduction():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 11.0                     # slowest rank's time
    assert r0[1] == r1[1] == r0[2] + r1[2]            # steps summed over ranks
    assert r0[3] != r1[3]                             # each rank has its own seeds


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(5.0, 123, None, "cpu") == (5.0, 123)
