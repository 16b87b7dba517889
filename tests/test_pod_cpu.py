"""Partition over data (pod.py) across CPU ranks (gloo, world size 2 and 3).

The exchange protocol of the paper's data-parallel mode is run by the
library's driver (pod.trace: round, all-to-all-v of the particles that left a
rank's bricks, sum reduction of the particles left, merge of the ranks'
partial line buffers) over real gloo process groups.  Each rank's advection
is a CPU stand-in built from the FP64 oracle's single steps, on a grid with
unit spacing (world = index space), so that the assembled lines must equal
the oracle's uninterrupted trace bit for bit: every vertex, length, status
and margin, with particles crossing ranks many times.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2606_02627_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    g = inputs.Grid((25, 21, 23), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    F = inputs.turbulence_field(g, inputs.turbulence_modes(51, n_modes=32, kmax=3)).numpy()
    seeds = inputs.uniform_seeds(g, 80, 51).astype(np.float64)
    seeds[:2] = -3.0                                       # OUT
    dt = 0.7 / oracle.max_speed(F, g.spacing)
    return g, F, seeds, dt, 120


class OracleEngine:
    """One rank: advects the particles in its own bricks with single oracle
    steps; records are (line, x, y, z, step) float64 rows."""

    def __init__(self, g, F, seeds, dt, max_steps, bricks, owner, rank, world):
        self.g, self.F, self.seeds, self.dt, self.ms = g, F, seeds, dt, max_steps
        self.bricks, self.owner, self.rank, self.world = bricks, owner, rank, world
        n = len(seeds)
        self.slab = torch.full((n, max_steps + 1, 3), float("inf"), dtype=torch.float64)
        self.length = torch.zeros(n, dtype=torch.int32)
        self.status = torch.zeros(n, dtype=torch.uint8)
        self.margin = torch.full((n,), float("inf"), dtype=torch.float64)
        self.queue = []

    def _rank_of(self, p):
        b = oracle.owner_brick(self.g.dims, self.bricks, p)
        return int(self.owner[(b[2] * self.bricks[1] + b[1]) * self.bricks[0] + b[0]])

    def begin(self):
        hi = np.asarray(self.g.dims, dtype=np.float64) - 1
        for i, p in enumerate(self.seeds):
            if not ((p >= 0).all() and (p <= hi).all()):
                self.status[i] = oracle.OUT
                continue
            self.slab[i, 0] = torch.from_numpy(p)
            self.length[i] = 1
            if self._rank_of(p) == self.rank:
                self.queue.append((i, p.copy(), 0))
        return len(self.queue)

    def round(self):
        out = [[] for _ in range(self.world)]
        queue, self.queue = self.queue, []
        for line, p, step in queue:
            while True:
                if step == self.ms:
                    self.status[line] = oracle.MAXSTEPS
                    self.length[line] = step + 1
                    break
                L = oracle.trace_streamlines(self.F, self.g.origin, self.g.spacing, p[None, :], self.dt, 1,
                                             nthreads=1)
                if L.length[0] < 2:
                    self.status[line] = int(L.status[0])
                    self.margin[line] = float(L.margin[0])
                    self.length[line] = step + 1
                    break
                p = L.line(0)[1].copy()
                step += 1
                self.slab[line, step] = torch.from_numpy(p)
                r = self._rank_of(p)
                if r != self.rank:
                    out[r].append([line, p[0], p[1], p[2], step])
                    break
        sends = [torch.from_numpy(np.frombuffer(np.asarray(o, dtype=np.float64).reshape(-1, 5).tobytes(),
                                                dtype=np.uint8).copy()) for o in out]
        return len(self.queue), sends

    def import_(self, records):
        rows = np.frombuffer(records.contiguous().numpy().tobytes(), dtype=np.float64).reshape(-1, 5)
        for r in rows:
            self.queue.append((int(r[0]), r[1:4].copy(), int(r[4])))

    def queued(self):
        return len(self.queue)

    def line_buffers(self):
        return {"slab": (self.slab, "min"), "length": (self.length, "max"), "status": (self.status, "max"),
                "margin": (self.margin, "min")}


def _worker(rank, world, port, bricks, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_02627_gb300 import pod
    g, F, seeds, dt, ms = _problem()
    owner = pod.partition_bricks(bricks, world)
    eng = OracleEngine(g, F, seeds, dt, ms, bricks, owner, rank, world)
    rounds = pod.trace(eng, pod.DistTransport())
    out[rank] = (rounds, eng.slab.numpy(), eng.length.numpy(), eng.status.numpy(), eng.margin.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,bricks", [(2, (2, 2, 2)), (3, (3, 1, 3))])
def test_pod_exchange_assembles_the_undivided_lines(world, bricks):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, bricks, out), nprocs=world, join=True)
    g, F, seeds, dt, ms = _problem()
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, ms)
    res = [out[r] for r in range(world)]
    assert all(r[0] == res[0][0] for r in res)             # every rank ran the same rounds
    assert res[0][0] > 3                                    # particles crossed ranks repeatedly
    for rounds, slab, length, status, margin in res:        # every rank holds the merged lines
        np.testing.assert_array_equal(length, ref.length)
        np.testing.assert_array_equal(status, ref.status)
        for i in range(len(seeds)):
            np.testing.assert_array_equal(slab[i, :length[i]], ref.line(i))
        stopped = np.isin(ref.status, (oracle.EXIT, oracle.STAGNANT))
        np.testing.assert_array_equal(margin[stopped], ref.margin[stopped])


def test_partition_bricks():
    from paper_2606_02627_gb300 import pod
    o = pod.partition_bricks((4, 4, 4), 2)
    assert o.tolist() == [0] * 32 + [1] * 32                 # z halves
    o = pod.partition_bricks((3, 1, 3), 3)
    assert sorted(set(o.tolist())) == [0, 1, 2] and np.all(np.diff(o) >= 0)
    with pytest.raises(ValueError):
        pod.partition_bricks((2, 1, 1), 3)
