"""Partition over data (POD) across ranks: the paper's data-parallel mode.

The bricks of the field are owned by ranks (one GPU each).  Every rank
uploads every seed and keeps those in its own bricks; each round it advects
its local particles, hands the particles that left its bricks to their
owners in one all-to-all-v exchange of 32-byte records, and all ranks stop
once a sum reduction finds no particle queued anywhere (RaFI's emitOutgoing /
all-to-all forwarding and the numActiveAcrossAllRanks test of Sec. 3.1.2 and
Listing 2).  Lines are then assembled by merging every rank's partial line
buffers: each vertex is written by the one rank that advected that step (the
others hold +inf), so an elementwise minimum over ranks is the line; lengths
and statuses merge by maximum (the rank where a line stopped wrote them),
margins by minimum.

Transport: ``torch.distributed`` (NCCL between GPUs, gloo on CPU) through
``DistTransport``; ``LocalTransport`` joins ranks that live in one process
(for instance several tracers on one GPU), with the same protocol.
"""
from __future__ import annotations

import numpy as np
import torch


def partition_bricks(bricks, world: int) -> np.ndarray:
    """Owner rank of every brick (linear index (bz*By + by)*Bx + bx): contiguous
    ranges of that index, i.e. slabs of z layers when world divides Bz."""
    nb = int(np.prod(bricks))
    if not 1 <= world <= min(nb, 64):
        raise ValueError(f"world {world} must be in [1, min(bricks, 64)]")
    return (np.arange(nb, dtype=np.int64) * world // nb).astype(np.int32)


class DistTransport:
    """Exchange over a torch.distributed process group."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        backend = dist.get_backend(group)
        self.device = torch.device(device) if device else (
            torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu"))

    def alltoallv(self, sends):
        """sends[r]: uint8 tensor for rank r; returns the tensors received from every rank."""
        d = self.dist
        counts = torch.tensor([int(x.numel()) for x in sends], dtype=torch.int64, device=self.device)
        rcounts = torch.empty_like(counts)
        d.all_to_all_single(rcounts, counts, group=self.group)
        rc = rcounts.tolist()
        out = torch.empty(sum(rc), dtype=torch.uint8, device=self.device)
        inp = torch.cat([x.to(self.device) for x in sends]) if sends else torch.empty(0, dtype=torch.uint8)
        d.all_to_all_single(out, inp, rc, counts.tolist(), group=self.group)
        return list(torch.split(out, rc))

    def sum(self, value: int) -> int:
        t = torch.tensor([int(value)], dtype=torch.int64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return int(t.item())

    def reduce_(self, tensor: torch.Tensor, op: str):
        """In-place elementwise min or max over ranks."""
        d = self.dist
        o = {"min": d.ReduceOp.MIN, "max": d.ReduceOp.MAX}[op]
        t = tensor if tensor.device == self.device else tensor.to(self.device)
        d.all_reduce(t, op=o, group=self.group)
        if t is not tensor:
            tensor.copy_(t)


class GpuEngine:
    """One rank's side of the exchange on a library tracer (api.Tracer)."""

    def __init__(self, tracer, brick_owner, rank: int, world: int):
        self.tr = tracer
        self.rank = rank
        self.world = world
        tracer.pod_setup(brick_owner, rank, world)

    def begin(self) -> int:
        return self.tr.pod_begin()

    def round(self):
        local, ex = self.tr.pod_round()
        return local, [self.tr.pod_export(r, int(ex[r])) for r in range(self.world)]

    def import_(self, records: torch.Tensor):
        self.tr.pod_import(records.to(self.tr.workspace.device))

    def queued(self) -> int:
        return self.tr.pod_queued()

    def line_buffers(self):
        slab, length, status, margin = self.tr.line_buffers()
        return {"slab": (slab, "min"), "length": (length, "max"), "status": (status, "max"), "margin": (margin, "min")}


def _merge(buffers, transport):
    for t, op in buffers.values():
        if t.dtype == torch.uint8:               # reduce as int32 (every backend reduces those)
            w = t.to(torch.int32)
            transport.reduce_(w, op)
            t.copy_(w.to(torch.uint8))
        else:
            transport.reduce_(t, op)


def trace(engine, transport, max_rounds: int = 1 << 30) -> int:
    """Runs the rounds of one rank until no rank has a particle queued, then
    merges the ranks' line buffers (every rank ends with the whole lines).
    Returns the number of rounds."""
    engine.begin()
    rounds = 0
    while transport.sum(engine.queued()) > 0:
        if rounds >= max_rounds:
            raise RuntimeError("round cap reached with particles left")
        _, exports = engine.round()
        received = transport.alltoallv(exports)
        engine.import_(torch.cat([r.to(received[0].device) for r in received]) if received else
                       torch.empty(0, dtype=torch.uint8))
        rounds += 1
    _merge(engine.line_buffers(), transport)
    return rounds


class LocalTransport:
    """Ranks that live in one process: trace_local drives them in lockstep."""

    @staticmethod
    def trace_local(engines, max_rounds: int = 1 << 30) -> int:
        world = len(engines)
        for e in engines:
            e.begin()
        rounds = 0
        while sum(e.queued() for e in engines) > 0:
            if rounds >= max_rounds:
                raise RuntimeError("round cap reached with particles left")
            outs = [e.round()[1] for e in engines]
            for r, e in enumerate(engines):
                parts = [outs[s][r] for s in range(world) if outs[s][r].numel()]
                if parts:
                    e.import_(torch.cat([p.to(parts[0].device) for p in parts]))
            rounds += 1
        bufs = [e.line_buffers() for e in engines]
        for key in bufs[0]:
            op = bufs[0][key][1]
            acc = bufs[0][key][0].clone()
            for b in bufs[1:]:
                t = b[key][0].to(acc.device)
                if op == "min":
                    torch.minimum(acc, t, out=acc)
                else:
                    torch.maximum(acc, t, out=acc)
            for b in bufs:
                b[key][0].copy_(acc)
        return rounds
