"""Serving loop: continuous batching of interactive seed-placement requests.

The paper's interactive application lets a user place seed regions while the
field stays resident and lines come back for display (Sec. 4).  Here requests
(a seed box or rake on one of several resident fields, with its own step cap)
arrive as a Poisson process; each is admitted into the running batch as soon
as line slots and slab memory allow, its particles share the persistent
kernel with every other admitted request, and its lines are read back and its
memory released as soon as its last line stops.  Latency is measured from
arrival to lines ready (host clock after the readback's stream synchronises).
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field as dfield

import numpy as np
import torch

from . import api, inputs


@dataclass
class Request:
    idx: int
    arrival: float                  # seconds after the start of serving
    field: int                      # index into the server's fields
    seeds: np.ndarray               # (n, 3) float32 world
    max_steps: int
    shape: str                      # "box" or "rake"
    rid: int | None = None
    admitted: float | None = None
    done: float | None = None
    lines: int = 0
    vertices: int = 0
    steps: int = 0
    result: object = dfield(default=None, repr=False)


@dataclass
class ResidentField:
    field: api.Field
    grid: inputs.Grid
    dt: float


def make_requests(fields, n_requests: int, rate_hz: float, seed: int, min_seeds=100, max_seeds=1_000_000,
                  min_steps=10, max_steps=5000, device_seeds=True) -> list:
    """Poisson arrivals (exponential gaps) at rate_hz; seed count and step cap
    log-uniform; box or rake with equal probability; field uniform.  Every
    random number derives from (seed, request index)."""
    u = inputs.uniform(seed, 20, 6 * n_requests).reshape(n_requests, 6)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += -math.log(1.0 - u[i, 0]) / rate_hz
        n = int(round(math.exp(math.log(min_seeds) + (math.log(max_seeds) - math.log(min_seeds)) * u[i, 1])))
        ms = int(round(math.exp(math.log(min_steps) + (math.log(max_steps) - math.log(min_steps)) * u[i, 2])))
        fi = min(len(fields) - 1, int(u[i, 3] * len(fields)))
        g = fields[fi].grid
        N = np.array(g.dims, dtype=np.float64) - 1
        r = inputs.uniform(seed * 1000003 + i, 21, 6)
        if u[i, 4] < 0.5:
            lo = r[:3] * 0.7 * N
            hi = lo + (0.05 + 0.25 * r[3:]) * N
            s = inputs.box_seeds(g, n, seed * 1000003 + i, lo, np.minimum(hi, N))
            shape = "box"
        else:
            a = (0.1 + 0.8 * r[:3]) * N
            b = (0.1 + 0.8 * r[3:]) * N
            s = inputs.rake_seeds(g, n, a, b)
            shape = "rake"
        reqs.append(Request(i, t, fi, s, ms, shape))
    return reqs


class Server:
    def __init__(self, ctx: api.Context, fields, max_lines: int, slab_bytes: int, layout="cell8",
                 rounds_per_launch: int = 2, max_requests: int = 1024, schedule=None):
        self.ctx = ctx
        self.fields = fields
        self.rounds = rounds_per_launch
        sched = schedule or {}
        self.batch = api.Batch(ctx, max_lines=max_lines, slab_bytes=slab_bytes, layout=layout,
                               max_requests=max_requests, max_fields=max(1, len(fields)),
                               max_bricks=max(1, sum(f.field.bricks[0] * f.field.bricks[1] * f.field.bricks[2]
                                                     for f in fields)), **sched)
        self.stream = torch.cuda.Stream(device=f"cuda:{ctx.device}")

    def _submit(self, r: Request) -> bool:
        f = self.fields[r.field]
        seeds = torch.from_numpy(r.seeds)
        rid = self.batch.submit(f.field, seeds, f.dt, r.max_steps, stream=self.stream)
        if rid is None:
            return False
        r.rid = rid
        return True

    def _retire(self, rid: int, by_rid: dict, t0: float, clock, readback: str, keep: bool):
        r = by_rid.pop(rid)
        lines = self.batch.get_lines(rid, device=readback, stream=self.stream)
        self.stream.synchronize()
        r.done = clock() - t0
        lens = (lines.offsets[1:] - lines.offsets[:-1]).cpu().numpy()
        r.lines = int(len(lens))
        r.vertices = int(lens.sum())
        r.steps = int(np.maximum(lens - 1, 0).sum())
        if keep:
            r.result = lines
        self.batch.release(rid, stream=self.stream)

    def serve(self, requests, readback="cuda", keep_results=False, clock=time.perf_counter, time_limit=600.0):
        """Runs the request stream to completion; returns the requests with
        admission / completion times and line counts filled in."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        by_rid = {}
        t0 = clock()
        while pending or waiting or by_rid:
            now = clock() - t0
            if now > time_limit:
                raise RuntimeError("serving exceeded its time limit")
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission in arrival order while memory allows (continuous batching)
            while waiting:
                r = waiting[0]
                if not self._submit(r):
                    if not by_rid:
                        raise RuntimeError(f"request {r.idx} ({len(r.seeds)} seeds x {r.max_steps} steps) "
                                           "can never fit the batch")
                    break
                waiting.popleft()
                r.admitted = clock() - t0
                by_rid[r.rid] = r
            if by_rid:
                self.batch.run(self.rounds, stream=self.stream)
                for rid in self.batch.finished(stream=self.stream):
                    self._retire(rid, by_rid, t0, clock, readback, keep_results)
            elif pending:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        return requests


def summarize(requests) -> dict:
    lat = np.array([r.done - r.arrival for r in requests])
    steps = sum(r.steps for r in requests)
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
            "particle_steps": int(steps), "makespan_s": float(span),
            "particle_steps_per_s": float(steps / span) if span > 0 else 0.0,
            "queue_ms_p99": float(np.percentile([(r.admitted - r.arrival) * 1e3 for r in requests], 99))}
