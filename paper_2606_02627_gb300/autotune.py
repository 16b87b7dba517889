"""Autotuner of the persistent advection kernel's structure and schedule.

Tunables:

* structure: the field layout (CELL8 cell records, run by the decoupled-lane
  kernel; TILED4 4x4x4 sample tiles and LINEAR samples, run by the lockstep
  kernel), the brick shape (bricks per axis) and the rounds policy (every
  brick each round, or brick-major windows of w bricks: sg_tracer_params
  .brick_window);
* schedule (all `sg_tracer_params` fields): threads per CTA, CTAs per SM of
  the persistent grid, steps a particle may take per round before it is
  re-queued in its own brick, and how far a round's end is cut short once its
  queue is empty (the library's drain default, or no limit).

The search is successive halving in two stages: the structures first, each
with the library's default schedule, then the schedules of the best
structures.  Every candidate traces a prefix of the seeds; the faster half
traces a four times larger prefix, and so on.  The winner is cached in a JSON
file keyed by the GPU, the storage type, the grid, the problem size and (when
the structure is not tuned) the layout and bricks, so a later run of the same
shape skips the search.  Every candidate computes the same lines: the
arithmetic of a particle does not depend on the schedule or the layout.

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
LAYOUTS = ("cell8", "tiled4", "linear")
DEFAULT_DECOUPLED = (256, 3, 1024, 0)         # the library's schedule of the decoupled-lane kernel
BRICKS = ((4, 4, 4), (2, 2, 2), (8, 8, 8))


def candidates(max_threads_per_sm: int = 2048, regs_limit_threads: int = 1024):
    """Grid of schedules (block_size, blocks_per_sm, steps_per_round, drain_steps)
    to try (drain_steps 0: the library default; -1: no limit).  Blocks of at
    most 256 threads: the kernels are built for that (their register budget)."""
    out = []
    for block, threads, spr, drain in itertools.product((64, 128, 256), (256, 384, 512, 768, 1024),
                                                         (256, 512, 1024, 2048), (0, -1)):
        if threads > min(max_threads_per_sm, regs_limit_threads) or threads % block:
            continue
        out.append((block, threads // block, spr, drain))
    return out


def structures(n_bricks_default: int = 64, layouts=LAYOUTS, bricks=BRICKS, windows=None):
    """Structures (layout, bricks, brick_window) to try: every layout and brick
    shape with all bricks advanced each round, plus brick-major windows of an
    eighth and of half the bricks for the first layout."""
    out = []
    for lay, br in itertools.product(layouts, bricks):
        out.append((lay, tuple(br), 0))
    nb = n_bricks_default
    for w in (windows if windows is not None else (max(1, nb // 8), max(1, nb // 2))):
        out.append((layouts[0], tuple(bricks[0]), int(w)))
    return out


def schedule_of(c) -> dict:
    """The sg_tracer_params fields of one schedule tuple."""
    sched = dict(block_size=c[0], blocks_per_sm=c[1], steps_per_round=c[2])
    if len(c) > 3:
        sched["drain_steps"] = c[3]
    return sched


def key_of(device: int, dtype, where: str, dims, n_seeds: int, max_steps: int) -> str:
    """Cache key: GPU name, storage type, layout and bricks (or "structure"
    when they are tuned too), grid, seeds (power of two below) and step cap."""
    name = torch.cuda.get_device_name(device)
    dt = api.DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return (f"{name}|{dt}|{where}|{'x'.join(map(str, dims))}|"
            f"seeds2^{int(math.log2(max(1, n_seeds)))}|steps{max_steps}")


def shape_key(field: api.Field, n_seeds: int, max_steps: int) -> str:
    return key_of(field.ctx.device, field.desc.dtype, f"{field.desc.layout}|{'x'.join(map(str, field.bricks))}",
                  field.dims, n_seeds, max_steps)


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


def _halving(cands, seeds, first, rounds, run, log, tag, keep=None):
    """Successive halving: every candidate runs on a prefix of the seeds, the
    faster half on a four times larger prefix.  run(candidate, prefix) -> ms.
    `keep` (the library's default) stays in every round, so that the last
    round, on the largest prefix, can only pick something at least as fast:
    small prefixes are dominated by the rounds' tails and can misjudge the
    full problem.  Returns (ranked candidates of the last round, history)."""
    cands = list(cands)
    if keep is not None and keep not in cands:
        cands.append(keep)
    n = min(first, int(seeds.shape[0]))
    history = []
    scored = []
    for r in range(rounds):
        prefix = seeds[:n].contiguous()
        scored = []
        for c in cands:
            ms = run(c, prefix)
            scored.append((ms, c))
            if log:
                log(f"autotune {tag} r{r} n={n} {c} {ms:.3f} ms")
        scored.sort(key=lambda x: x[0])
        history.append([(ms, list(c) if isinstance(c, tuple) else c, n) for ms, c in scored])
        if len(scored) <= 1 or n >= seeds.shape[0]:
            break
        cands = [c for _, c in scored[:max(1, len(scored) // 2)]]
        if keep is not None and keep not in cands:
            cands.append(keep)
        n = min(int(seeds.shape[0]), n * 4)
    return [c for _, c in scored], history


def _load(cache):
    if cache and os.path.exists(cache):
        try:
            return json.load(open(cache))
        except (OSError, ValueError):
            return {}
    return {}


def _store(cache, db, key, entry):
    if not cache:
        return
    os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
    db[key] = entry
    tmp = cache + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, cache)


def tune(ctx: api.Context, field: api.Field, seeds: torch.Tensor, dt: float, max_steps: int,
         cands=None, first: int = 1 << 16, rounds: int = 3, cache: str | None = DEFAULT_CACHE,
         stream=None, log=None, keep=None) -> dict:
    """The fastest schedule {block_size, blocks_per_sm, steps_per_round, drain_steps}
    for this field as it is (its layout and bricks)."""
    key = shape_key(field, int(seeds.shape[0]), max_steps)
    db = _load(cache)
    if key in db:
        return dict(db[key]["schedule"])
    stream = stream or torch.cuda.current_stream()
    t_start = time.time()

    def run(c, prefix):
        tr = api.Tracer(ctx, field, capacity=prefix.shape[0], dt=dt, max_steps=max_steps, **schedule_of(c))
        _time_trace(tr, prefix, stream)            # warm the graph
        ms = _time_trace(tr, prefix, stream)
        tr.close()
        return ms

    ranked, history = _halving(cands or candidates(), seeds, first, rounds, run, log, "schedule", keep=keep)
    sched = schedule_of(ranked[0])
    _store(cache, db, key, {"schedule": sched, "history": history, "seconds": time.time() - t_start})
    return sched


def tune_structure(ctx: api.Context, source: torch.Tensor, grid, dtype: str, seeds: torch.Tensor, dt: float,
                   max_steps: int, structs=None, cands=None, first: int = 1 << 14, rounds: int = 3,
                   finalists: int = 2, cache: str | None = DEFAULT_CACHE, stream=None, log=None) -> dict:
    """The fastest structure and schedule for a field given as a global FP32
    array `source` ([nz][ny][nx][3] on the device) on `grid`, stored as
    `dtype`: returns {"layout", "bricks", "brick_window", "schedule"}.  Stage 1
    halves the structures (layout, bricks, window) under the default schedule;
    stage 2 halves the schedules of the `finalists` best structures."""
    key = key_of(ctx.device, dtype, "structure", grid.dims, int(seeds.shape[0]), max_steps)
    db = _load(cache)
    if key in db:
        return dict(db[key]["choice"])
    stream = stream or torch.cuda.current_stream()
    t_start = time.time()
    fields = {}

    def field_of(layout, bricks):
        k = (layout, tuple(bricks))
        if k not in fields:
            # one field at a time: a structure's field is dropped when the next is built
            fields.clear()
            torch.cuda.empty_cache()
            f = api.Field(ctx, grid.dims, grid.origin, grid.spacing, bricks=bricks, dtype=dtype, layout=layout)
            f.set_global(source, stream=stream)
            fields[k] = f
        return fields[k]

    def run_structure(s, prefix, sched=None):
        layout, bricks, window = s
        fld = field_of(layout, bricks)
        tr = api.Tracer(ctx, fld, capacity=prefix.shape[0], dt=dt, max_steps=max_steps, brick_window=window,
                        **(sched or {}))
        _time_trace(tr, prefix, stream)
        ms = _time_trace(tr, prefix, stream)
        tr.close()
        return ms

    structs = list(structs or structures())
    # stage 1: structures under the library's default schedule (brick-window
    # candidates beyond the field's bricks advance every brick: skipped)
    structs = [s for s in structs if s[2] == 0 or s[2] < s[1][0] * s[1][1] * s[1][2]]
    # group by field so that each field is built once per halving round
    default_struct = ("cell8", (4, 4, 4), 0)
    ranked_s, hist_s = _halving(sorted(structs), seeds, first, rounds, lambda s, p: run_structure(s, p), log,
                                "structure", keep=default_struct if default_struct in structs else None)
    best = ranked_s[:max(1, finalists)]
    # stage 2: schedules of the best structures
    pairs = [(s, c) for s in best for c in (cands or candidates())]
    pairs.sort(key=lambda x: (x[0][0], x[0][1]))
    # the library's schedule of the decoupled-lane kernel: 3 CTAs of 256, 1024 steps per round, its drain
    default_pair = (default_struct, DEFAULT_DECOUPLED)
    ranked_p, hist_p = _halving(pairs, seeds, first, rounds,
                                lambda sc, p: run_structure(sc[0], p, schedule_of(sc[1])), log, "schedule",
                                keep=default_pair if default_struct in structs else None)
    (layout, bricks, window), c = ranked_p[0]
    choice = {"layout": layout, "bricks": list(bricks), "brick_window": int(window), "schedule": schedule_of(c)}
    fields.clear()
    torch.cuda.empty_cache()
    _store(cache, db, key, {"choice": choice, "history": {"structure": hist_s, "schedule": hist_p},
                            "seconds": time.time() - t_start})
    return choice
