"""Schedule autotuner of the persistent advection kernel.

Tunables (all `sg_tracer_params` fields): threads per CTA, CTAs per SM of the
persistent grid, steps a particle may take per round before it is re-queued
in its own brick, and whether a round's end is cut short once its queue is
empty (the library's drain default, or no limit).  The search is successive halving: every
candidate traces a small prefix of the seeds, the faster half traces a larger
prefix, and so on; the winner is cached in a JSON file keyed by the GPU, the
field's storage type / layout / size / bricks and the problem size, so a
later run of the same shape skips the search.

Timing is by CUDA events on the tracer's stream around `sg_tracer_trace`
(the production graph launch); every candidate traces the same seeds.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time

import torch

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "streamgb", "autotune.json")


def candidates(max_threads_per_sm: int = 2048, regs_limit_threads: int = 1024):
    """Grid of (block_size, blocks_per_sm, steps_per_round, drain_steps) to try
    (drain_steps 0: the library default; -1: no limit)."""
    out = []
    for block, threads, spr, drain in itertools.product((64, 128, 256), (256, 384, 512, 768, 1024), (128, 256, 512),
                                                         (0, -1)):
        if threads > min(max_threads_per_sm, regs_limit_threads) or threads % block:
            continue
        out.append((block, threads // block, spr, drain))
    return out


def schedule_of(c) -> dict:
    """The sg_tracer_params fields of one candidate tuple."""
    sched = dict(block_size=c[0], blocks_per_sm=c[1], steps_per_round=c[2])
    if len(c) > 3:
        sched["drain_steps"] = c[3]
    return sched


def shape_key(field: api.Field, n_seeds: int, max_steps: int) -> str:
    name = torch.cuda.get_device_name(field.ctx.device)
    return (f"{name}|{field.desc.dtype}|{field.desc.layout}|{'x'.join(map(str, field.dims))}|"
            f"{'x'.join(map(str, field.bricks))}|seeds2^{int(math.log2(max(1, n_seeds)))}|steps{max_steps}")


def _time_trace(tr: api.Tracer, seeds: torch.Tensor, stream) -> float:
    tr.upload_seeds(seeds, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tr.trace(stream=stream)
    e1.record(stream)
    e1.synchronize()
    tr.check(stream=stream)
    return e0.elapsed_time(e1)


def tune(ctx: api.Context, field: api.Field, seeds: torch.Tensor, dt: float, max_steps: int,
         cands=None, first: int = 1 << 16, rounds: int = 3, cache: str | None = DEFAULT_CACHE,
         stream=None, log=None) -> dict:
    """Returns the fastest {block_size, blocks_per_sm, steps_per_round, drain_steps} for this shape."""
    key = shape_key(field, int(seeds.shape[0]), max_steps)
    db = {}
    if cache and os.path.exists(cache):
        try:
            db = json.load(open(cache))
        except (OSError, ValueError):
            db = {}
        if key in db:
            return dict(db[key]["schedule"])
    stream = stream or torch.cuda.current_stream()
    cands = list(cands or candidates())
    n = min(first, int(seeds.shape[0]))
    history = []
    t_start = time.time()
    for r in range(rounds):
        prefix = seeds[:n].contiguous()
        scored = []
        for c in cands:
            sched = schedule_of(c)
            tr = api.Tracer(ctx, field, capacity=n, dt=dt, max_steps=max_steps, **sched)
            _time_trace(tr, prefix, stream)            # warm the graph
            ms = _time_trace(tr, prefix, stream)
            tr.close()
            del tr
            scored.append((ms, c))
            if log:
                log(f"autotune r{r} n={n} {c} {ms:.3f} ms")
        scored.sort()
        history.append([(ms, list(c), n) for ms, c in scored])
        cands = [c for _, c in scored[:max(1, len(scored) // 2)]]
        if len(cands) == 1 or n >= seeds.shape[0]:
            break
        n = min(int(seeds.shape[0]), n * 4)
    sched = schedule_of(cands[0])
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        db[key] = {"schedule": sched, "history": history, "seconds": time.time() - t_start}
        tmp = cache + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return sched
