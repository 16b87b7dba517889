#!/usr/bin/env python3
"""Benchmark: RK4 particle-steps/s of brick-decomposed steady streamlines.

Workload (one step = the whole hot path on one batch): a 512^3 FP32 vec3
synthetic-turbulence field (256 divergence-free Fourier modes, |k|^-5/3
amplitudes, SplitMix64 seed 1) resident in HBM is cut into 4x4x4 bricks with a
one-cell ghost shell and encoded to the benchmarked storage type; 1M seeds
(uniform over the grid) are uploaded and binned into per-brick queues; RK4
with h = 0.5 cell runs to max 2000 steps (exit / |v| < 1e-6 / cap) with
cross-brick hand-off queues; the lines are compacted to CSR.

`value` is the persistent form on the FP32 field (the samples as given, in
8-corner cell records), run by the decoupled-lane kernel.  The compact
storage forms (FX21: 21-bit fixed point, three components in 8 bytes with a
per-brick scale; BF16; FP16), the same FP32 field under the lockstep
persistent kernel, the plain FP32 per-seed kernel and (optionally) the
one-launch-per-step kernel of Listing 1 are timed in the same run under
`variants`.  `e2e` repeats the headline through the C ABI with the seeds
copied from page-locked host memory and the CSR lines copied to page-locked
host memory inside the timed region; each step's copy to the host runs on the
tracer's copy stream and overlaps the next step (sg_tracer_get_lines_overlapped),
and the timed region ends after the last step's copy.

Multi-GPU (torchrun): every rank traces its own 1M seeds on its own copy of the
field (independent work, weak scaling); only the timing barrier and the
max-over-ranks reduction cross ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes per particle-step: 4 samples x 8 corners x 3 components x element bytes + a 12-B vertex
# (FX21 packs 3 components in 8 bytes: 8/3 bytes per component, the same 64 bits per corner as BF16x4)
GATHER_BYTES = {"f32": 4 * 8 * 3 * 4 + 12, "bf16": 4 * 8 * 3 * 2 + 12, "f16": 4 * 8 * 3 * 2 + 12,
                "fx21": 4 * 8 * 8 + 12}
METRIC = "RK4 particle-steps/s"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512, help="samples per axis")
    ap.add_argument("--seeds", type=int, default=1 << 20)
    ap.add_argument("--max-steps", type=int, default=2000)
    ap.add_argument("--h", type=float, default=0.5)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16", "fx21"])
    ap.add_argument("--kernel", default="persistent", choices=["persistent", "lockstep"],
                    help="headline kernel: decoupled lanes (persistent, CELL8) or lanes in lockstep")
    ap.add_argument("--layout", default="cell8")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--per-step", action="store_true", help="also time the one-launch-per-step kernel")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle baseline")
    ap.add_argument("--schedule", default="", help="block,blocks_per_sm,steps_per_round[,drain_steps]")
    ap.add_argument("--requests", type=int, default=160, help="serve: requests in the Poisson stream")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end pass through host buffers (large workloads whose CSR would not fit a "
                         "page-locked host buffer)")
    ap.add_argument("--config", default="steady",
                    choices=["steady", "streak", "serve", "umesh", "plain", "bidir", "path", "pod"],
                    help="steady: brick-decomposed streamlines (the headline); streak: unsteady streaklines with "
                         "time slices streamed from page-locked host memory; bidir, path, pod: bidirectional "
                         "lines from a seed shape, path lines, partition over data (ranks emulated on one GPU)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the rounds from the host (sg_tracer_trace_timed) instead of the CUDA graph, so that "
                         "a profiler sees every advection-kernel launch")
    ap.add_argument("--once", action="store_true",
                    help="profiling case: one step of the headline form, then print its particle-steps and exit")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the headline on the library's default structure and schedule instead of the "
                         "autotuner's pick (layout, bricks, brick window, threads, CTAs/SM, steps per round, drain)")
    ap.add_argument("--serve-requests", type=int, default=96,
                    help="requests of the short serving run whose latency the headline line reports (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    """Hash of the advection kernels' sources.  The host-side tracer state
    (struct sg_tracer in tracer.cuh), which no kernel reads, is left out."""
    h = hashlib.sha256()
    for f in ("advect.cu", "rk4.cuh", "common.cuh", "tracer.cuh"):
        src = open(os.path.join(ROOT, "paper_2606_02627_gb300", "csrc", f), "rb").read()
        if f == "tracer.cuh":
            src = re.sub(rb"\nstruct sg_tracer \{.*?\n\};\n", b"\n", src, count=1, flags=re.S)
        h.update(src)
    return h.hexdigest()[:16]


def counters(dtype, tag):
    """Per-particle-step counters of the advection kernel (tag "async": the
    decoupled-lane kernel, "lockstep": lanes in lockstep) from the committed
    ncu summary profiles/round_<tag>_<dtype>_traffic.txt, as {name: float},
    or {} if it is missing or the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", f"round_{tag}_{dtype}_traffic.txt")
    if not os.path.exists(p):
        return {}
    kv = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_hash():
        return {}
    out = {}
    for k, v in kv.items():
        try:
            out[k] = float(v)
        except ValueError:
            pass
    return out


def traffic_per_step(dtype, tag):
    """DRAM bytes per particle-step (committed ncu summary), or None."""
    return counters(dtype, tag).get("dram_bytes_per_particle_step")


def issue_roofline(steps_per_s, thread_inst_per_step, sm_count, sm_mhz):
    """Instruction-issue bound of a kernel: each of an SM's 4 schedulers issues
    at most one warp instruction (32 threads' work) per cycle, so the peak is
    sm_count x 4 x 32 thread instructions per cycle.  achieved = the kernel's
    thread instructions per particle-step (ncu) x its particle-steps/s; the
    fraction counts both idle issue slots and idle lanes of a warp."""
    peak = sm_count * 4 * 32 * sm_mhz * 1e6
    achieved = thread_inst_per_step * steps_per_s
    return achieved / 1e9, peak / 1e9, achieved / peak


def copy_rates(dev, nbytes=1 << 31):
    """Page-locked host <-> device copy rates (GB/s) of one nbytes copy each way, CUDA events."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            with torch.cuda.stream(s):
                dst.copy_(src, non_blocking=True)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = nbytes / (best / 1e3) / 1e9
    del h, d
    return out


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def rank_seed(base: int, rank: int) -> int:
    """Seed stream of a rank: every rank traces its own seeds (weak scaling)."""
    return base + 1000 * rank


def reduce_over_ranks(ms: float, steps: int, dist, device):
    """Whole-job timing across ranks: the slowest rank's time and the sum of
    particle-steps (no collective on the data path: only these two numbers)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, steps
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([steps], dtype=torch.int64, device=device)
    dist.all_reduce(s)
    return float(t.item()), int(s.item())


def cpu_oracle_rate(F_host, grid, seeds, dt, max_steps, seconds, nthreads=None, n_seeds=None):
    """Oracle particle-steps/s on the host cores (all of them unless nthreads is given) over a bounded
    prefix of the seeds: sized to take about `seconds`, or the first n_seeds when given."""
    import oracle
    nthreads = nthreads or oracle.default_threads()
    if n_seeds:
        t = time.perf_counter()
        L = oracle.trace_streamlines(F_host, grid.origin, grid.spacing, seeds[:n_seeds], dt, max_steps, eps=1e-6,
                                     nthreads=nthreads)
        t0 = time.perf_counter() - t
        steps = int(L.steps().sum())
        return steps / t0, nthreads, n_seeds, steps, t0
    n0 = min(len(seeds), max(nthreads * 8, 64))
    t = time.perf_counter()
    L = oracle.trace_streamlines(F_host, grid.origin, grid.spacing, seeds[:n0], dt, max_steps, eps=1e-6,
                                 nthreads=nthreads)
    t0 = time.perf_counter() - t
    n = n0
    # a small calibration run overestimates the time per seed (start-up, load imbalance): rescale until
    # the sample takes at least half the target, at most three times
    for _ in range(3):
        if t0 >= 0.5 * seconds or n >= len(seeds):
            break
        n = int(min(len(seeds), max(n + 1, n * seconds / max(t0, 1e-3))))
        t = time.perf_counter()
        L = oracle.trace_streamlines(F_host, grid.origin, grid.spacing, seeds[:n], dt, max_steps, eps=1e-6,
                                     nthreads=nthreads)
        t0 = time.perf_counter() - t
    steps = int(L.steps().sum())
    return steps / t0, nthreads, n, steps, t0


def run_umesh(args, rank, world, local):
    """Unstructured field: the cells of a 128^3 grid of the synthetic turbulence (seed 1, 256 modes, |k| <= 16
    on [0, 2pi]^3) as 2,097,152 hexahedra with interior vertices jittered by up to 0.1 cell (the paper's
    galaxy-as-hexahedra variant, synthetic); 262,144 seeds, RK4 h = 0.5 cell, max 1000 steps, in rounds of at
    most 128 steps per particle; cells located by face walks and the BVH.  Step = trace + CSR compaction (the
    mesh is built once)."""
    import numpy as np
    import torch
    from paper_2606_02627_gb300 import api, inputs
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    ctx = api.Context(local)
    n = 129
    g = inputs.cube_grid(n)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1), device=dev).cpu().numpy()
    t0 = time.time()
    m = inputs.grid_mesh(g, F, kind="hex", jitter=0.1, seed=1)
    mesh = api.UMesh(ctx, m)
    build_s = time.time() - t0
    probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(1, 1, 1))
    probe.set_global(torch.from_numpy(F).to(dev))
    dt = args.h / probe.max_speed()
    del probe
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 1 << 18, rank_seed(1, rank), lo_cells=1.0)).to(dev)
    ms_steps, steps_total = 1000, 0
    for _ in range(args.warmup):
        mesh.trace(seeds, dt, ms_steps)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        lines = mesh.trace(seeds, dt, ms_steps)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    steps_total = int((lines.lengths().clamp(min=1) - 1).sum().item())
    out = {"metric": "RK4 particle-steps/s (unstructured hexahedra)", "value": steps_total / (ms / 1e3),
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": "unstructured: 128^3 grid cells of turbulence (seed 1) as 2,097,152 jittered "
                                  "hexahedra, BVH point location, 262144 seeds, RK4 h=0.5 cell, max 1000 steps",
                      "cells": mesh.n_cells, "mesh_build_s": build_s,
                      "mesh_device_bytes": int(mesh.workspace.numel()),
                      "mesh_bytes_per_cell": round(mesh.workspace.numel() / max(1, mesh.n_cells), 1),
                      "mean_steps_per_line": round(steps_total / seeds.shape[0], 1)},
           "particle_steps_per_step": steps_total}
    print(json.dumps(out))


def run_streak(args, rank, world, local):
    """Unsteady streaklines: 64 time slices of a 256^3 FP32 field (phases advancing in time, seed 3) in
    page-locked host memory, streamed one slice per step into three resident slots on a side stream;
    4096 release points (64 rakes x 64 points) each release one particle per step for 64 steps."""
    import numpy as np
    import torch
    from paper_2606_02627_gb300 import api, inputs
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    n, n_slices, rakes, per_rake = 256, 64, 64, 64
    g = inputs.cube_grid(n)
    modes = inputs.turbulence_modes(3)
    ctx = api.Context(local)
    host = torch.empty((n_slices, n, n, n, 3), dtype=torch.float32).pin_memory()
    vref = 0.0
    for s in range(n_slices):
        F = inputs.turbulence_field(g, modes, time_slice=s, n_slices=n_slices, device=dev)
        sp = torch.tensor(g.spacing, device=dev, dtype=torch.float32)
        vref = max(vref, float((F / sp).norm(dim=-1).max()))
        host[s].copy_(F)
        del F
    dt = args.h / vref
    # rakes: segments between two uniform points in the interior, 64 release points each
    u = inputs.uniform(3 + 1000 * rank, 9, rakes * 6).reshape(rakes, 6)
    a = 8 + (n - 17) * u[:, :3]
    b = 8 + (n - 17) * u[:, 3:]
    rel = np.concatenate([inputs.rake_seeds(g, per_rake, a[r], b[r]) for r in range(rakes)])
    rel_dev = torch.from_numpy(rel).to(dev)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(2, 2, 2), dtype="f32", layout="linear", n_slots=3,
                    slice_dt=dt)
    tr = api.Tracer(ctx, fld, capacity=len(rel), dt=dt, mode="streakline", inject_steps=per_rake)
    main_s = torch.cuda.Stream(device=dev)
    side = torch.cuda.Stream(device=dev)

    def run_once():
        fld.stream_slice(0, host[0], stream=side)
        fld.stream_slice(1, host[1], stream=side)
        tr.upload_seeds(rel_dev, stream=main_s)
        for j in range(1, n_slices):
            if j + 1 < n_slices:
                fld.stream_slice(j + 1, host[j + 1], stream=side)
            tr.step(1, sync=False, stream=main_s)
        tr.sizes(stream=main_s)                 # CSR scan of the streaklines

    run_once()
    torch.cuda.synchronize(dev)
    steps = tr.total_steps(stream=main_s)
    for _ in range(args.warmup):
        run_once()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(side)
    for _ in range(args.steps):
        run_once()
    main_s.wait_stream(side)
    e1.record(main_s)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    nl, nv = tr.sizes(stream=main_s)
    h2d = n_slices * n ** 3 * 12
    out = {"metric": "RK4 particle-steps/s (streaklines)", "value": steps / (ms / 1e3), "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": f"streaklines: {n_slices} slices of {n}^3 FP32 turbulence (seed 3) streamed from "
                                  f"page-locked host memory, {rakes * per_rake} release points x {per_rake} releases, "
                                  f"RK4 h={args.h} cell", "slots": 3, "bricks": "2x2x2"},
           "particle_steps_per_step": steps, "h2d_bytes_per_step": h2d, "h2d_gbs": h2d / (ms / 1e3) / 1e9,
           "streaklines": nl, "vertices": nv}
    print(json.dumps(out))


SERVE_WORKLOAD = ("serving: 8 resident fields {64,128,256,512}^3 x {FP32,BF16} turbulence (seeds 4-10), CELL8, "
                  "4x4x4 bricks; Poisson requests of 100-1M seeds (box/rake), max steps 10-5000, rate = 70 % of "
                  "the capacity measured on the same requests arriving at once")


def serve_workload(ctx, dev, n_requests, h, rank=0, tune=False):
    """Batched serving of interactive seed placement: 8 resident fields ({64,128,256,512}^3 x {FP32, BF16},
    synthetic turbulence, CELL8 layout, 4x4x4 bricks), Poisson requests of 100 to 1M seeds (box or rake),
    max steps 10-5000, admitted into one continuously batched persistent launch by free memory; the arrival
    rate is 70 % of the capacity measured on the same requests arriving at once.  Returns the statistics."""
    import torch
    from paper_2606_02627_gb300 import api, inputs, serving
    fields = []
    seed = 4
    for n in (64, 128, 256, 512):
        g = inputs.cube_grid(n)
        F = inputs.turbulence_field(g, inputs.turbulence_modes(seed), device=dev)
        probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4), dtype="f32")
        probe.set_global(F)
        dt = h / probe.max_speed()
        probe.close()
        del probe
        for dtype in ("f32", "bf16"):
            fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4), dtype=dtype, layout="cell8")
            fld.set_global(F)
            fields.append(serving.ResidentField(fld, g, dt))
        del F
        seed += 2
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    sched = None
    if tune:
        # the autotuner's pick on the largest FP32 field (a 64k-seed sample, cached per shape)
        from paper_2606_02627_gb300 import autotune
        big = fields[6]
        sample = torch.from_numpy(inputs.uniform_seeds(big.grid, 1 << 16, 99)).to(dev)
        sched = autotune.tune(ctx, big.field, sample, big.dt, 1000, first=1 << 14,
                              cache=os.path.join(tempfile.gettempdir(), "streamgb_autotune.json"))
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(dev)
    slab = int(min(free * 0.6, 160e9))
    srv = serving.Server(ctx, fields, max_lines=8 << 20, slab_bytes=slab, rounds_per_launch=2,
                         max_requests=1024, schedule=sched)
    base = serving.make_requests(fields, n_requests, rate_hz=1.0, seed=4 + 1000 * rank)
    # capacity: the same requests all arriving at once
    burst = [serving.Request(r.idx, 0.0, r.field, r.seeds, r.max_steps, r.shape) for r in base]
    srv.serve(burst)
    cap = serving.summarize(burst)
    rate = 0.7 * len(burst) / cap["makespan_s"]
    reqs = [serving.Request(r.idx, r.arrival / rate, r.field, r.seeds, r.max_steps, r.shape) for r in base]
    srv.serve(reqs)
    st = serving.summarize(reqs)
    out = {"requests": len(reqs), "rate_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
           "max_ms": st["max_ms"], "particle_steps_per_s": st["particle_steps_per_s"],
           "particle_steps": st["particle_steps"], "queue_ms_p99": st["queue_ms_p99"],
           "capacity": {"requests_per_s": len(burst) / cap["makespan_s"],
                        "particle_steps_per_s": cap["particle_steps_per_s"]},
           "rounds_per_launch": 2, "slab_pool_bytes": slab, "schedule": sched or "library default"}
    del srv, fields
    torch.cuda.empty_cache()
    return out


def _cuda_ms(fn, steps, warmup, stream):
    """Mean ms of fn() over `steps` calls after `warmup`, by CUDA events on `stream`."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _turbulence_512(ctx, dev, args):
    """The headline's field: 512^3 synthetic turbulence (seed 1) on [0, 2pi]^3, with dt for h cells."""
    import torch
    from paper_2606_02627_gb300 import api, inputs
    g = inputs.cube_grid(512)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1), device=dev)
    probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4), dtype="f32")
    probe.set_global(F)
    dt = args.h / probe.max_speed()
    probe.close()
    torch.cuda.synchronize(dev)
    return g, F, dt


def run_bidir(args, rank, world, local):
    """Bidirectional lines from a seed shape: on the headline's field (512^3 turbulence, 4x4x4 bricks,
    CELL8 FP32), 1,048,576 seeds drawn on the device uniformly in the box of index [8, 503]^3
    (sg_seeds_box, SplitMix64 seed 1), each traced forward and backward up to 1000 steps (RK4, h = 0.5
    cell) and the two halves joined through the seed (sg_tracer_get_joined) into device buffers.
    Step = seed kernel + upload + trace + join."""
    import torch
    from paper_2606_02627_gb300 import api
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    ctx = api.Context(local)
    g, F, dt = _turbulence_512(ctx, dev, args)
    n_seeds, max_steps = 1 << 20, 1000
    lo = [g.origin[a] + 8 * g.spacing[a] for a in range(3)]
    hi = [g.origin[a] + (g.dims[a] - 9) * g.spacing[a] for a in range(3)]
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4), dtype="f32", layout="cell8")
    fld.set_global(F)
    del F
    tr = api.Tracer(ctx, fld, capacity=n_seeds, dt=dt, max_steps=max_steps, direction="both")
    stream = torch.cuda.Stream(device=dev)
    seeds = api.seeds_box(lo, hi, n_seeds, rank_seed(1, rank), stream=stream)
    tr.upload_seeds(seeds, stream=stream)
    tr.trace(stream=stream)
    J = tr.get_joined(stream=stream)
    stream.synchronize()
    off, vert, sv = torch.empty_like(J.offsets), torch.empty_like(J.vertices), torch.empty_like(J.seed_vertex)

    def step():
        sd = api.seeds_box(lo, hi, n_seeds, rank_seed(1, rank), stream=stream)
        tr.upload_seeds(sd, stream=stream)
        tr.trace(stream=stream)
        api.call("sg_tracer_get_joined", tr.h, None, None, api._ptr(off), api._ptr(vert), api._ptr(sv),
                 api._stream(stream))

    ms = _cuda_ms(step, args.steps, args.warmup, stream)
    steps = tr.total_steps(stream=stream)
    tr.check(stream=stream)
    out = {"metric": METRIC + " (bidirectional lines)", "value": steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "bidirectional: 512^3 FP32 turbulence (seed 1), 4x4x4 bricks, CELL8; 1048576 "
                                  "seeds uniform in index box [8, 503]^3 drawn on the device (sg_seeds_box), each "
                                  "traced forward and backward up to 1000 steps, RK4 h=0.5 cell, halves joined "
                                  "through the seed", "lines": 2 * n_seeds},
           "particle_steps_per_step": steps, "joined_vertices": int(J.vertices.shape[0])}
    print(json.dumps(out))


def run_path(args, rank, world, local):
    """Path lines: every seed released once at time 0 and followed through the unsteady field of the
    streakline workload (64 time slices of 256^3 FP32 turbulence, seed 3, streamed from page-locked host
    memory into three resident slots on a side stream), 1,048,576 seeds uniform in the interior (seed 3),
    RK4 h = 0.5 cell (dt = the slice interval), 63 steps with the field linear in time between slices.
    Step = the 64 slice uploads + seeds + 63 advection steps + the CSR of the lines in device buffers."""
    import torch
    from paper_2606_02627_gb300 import api, inputs
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    n, n_slices, n_seeds = 256, 64, 1 << 20
    g = inputs.cube_grid(n)
    modes = inputs.turbulence_modes(3)
    ctx = api.Context(local)
    host = torch.empty((n_slices, n, n, n, 3), dtype=torch.float32).pin_memory()
    vref = 0.0
    sp = torch.tensor(g.spacing, device=dev, dtype=torch.float32)
    for s_ in range(n_slices):
        F = inputs.turbulence_field(g, modes, time_slice=s_, n_slices=n_slices, device=dev)
        vref = max(vref, float((F / sp).norm(dim=-1).max()))
        host[s_].copy_(F)
        del F
    dt = args.h / vref
    steps_cap = n_slices - 1
    seeds = torch.from_numpy(inputs.uniform_seeds(g, n_seeds, rank_seed(3, rank), lo_cells=1.0)).to(dev)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(2, 2, 2), dtype="f32", layout="linear", n_slots=3,
                    slice_dt=dt)
    tr = api.Tracer(ctx, fld, capacity=n_seeds, dt=dt, max_steps=steps_cap, mode="pathline")
    main_s = torch.cuda.Stream(device=dev)
    side = torch.cuda.Stream(device=dev)
    nl, nv = [0], [0]
    bufs = {}

    def run_once():
        fld.stream_slice(0, host[0], stream=side)
        fld.stream_slice(1, host[1], stream=side)
        tr.upload_seeds(seeds, stream=main_s)
        for j in range(steps_cap):
            # step j+1 spans times j dt .. (j+1) dt: it needs slices j and j+1
            if j + 2 < n_slices:
                fld.stream_slice(j + 2, host[j + 2], stream=side)
            tr.step(1, sync=False, stream=main_s)
        if bufs:
            api.call("sg_tracer_get_lines", tr.h, None, None, api._ptr(bufs["off"]), api._ptr(bufs["v"]),
                     api._ptr(bufs["st"]), None, None, api._stream(main_s))

    run_once()
    torch.cuda.synchronize(dev)
    nl[0], nv[0] = tr.sizes(stream=main_s)
    bufs.update(off=torch.empty(nl[0] + 1, dtype=torch.int64, device=dev),
                v=torch.empty((max(nv[0], 1), 3), dtype=torch.float32, device=dev),
                st=torch.empty(max(nl[0], 1), dtype=torch.uint8, device=dev))
    steps = tr.total_steps(stream=main_s)

    def timed_once():
        run_once()
        main_s.wait_stream(side)

    ms = _cuda_ms(timed_once, args.steps, args.warmup, main_s)
    h2d = n_slices * n ** 3 * 12
    out = {"metric": METRIC + " (path lines)", "value": steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"path lines: {n_slices} slices of {n}^3 FP32 turbulence (seed 3) streamed from "
                                  f"page-locked host memory, {n_seeds} seeds released at t=0, {steps_cap} steps, "
                                  f"RK4 h={args.h} cell, field linear in time", "slots": 3, "bricks": "2x2x2",
                      "layout": "linear"},
           "particle_steps_per_step": steps, "h2d_bytes_per_step": h2d, "h2d_gbs": h2d / (ms / 1e3) / 1e9,
           "lines": nl[0], "vertices": nv[0]}
    print(json.dumps(out))


def run_pod(args, rank, world, local):
    """Partition over data with its ranks emulated on one GPU: the headline's field (512^3 turbulence,
    4x4x4 bricks, CELL8 FP32), 262,144 seeds uniform (seed 1), max 1000 steps, RK4 h = 0.5 cell; the 64
    bricks split over 4 ranks (pod.partition_bricks), one tracer per rank advancing only its own
    particles and handing the others to their owners between rounds (sg_tracer_pod_*, device copies
    between the ranks' buffers), then the ranks' lines merged.  Timed beside the undivided trace of the
    same seeds: the ratio is what the exchange costs when every rank shares one GPU."""
    import torch
    from paper_2606_02627_gb300 import api, pod
    from paper_2606_02627_gb300 import build as _build
    from paper_2606_02627_gb300 import inputs
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    ctx = api.Context(local)
    g, F, dt = _turbulence_512(ctx, dev, args)
    n_seeds, max_steps, ranks = 1 << 18, 1000, 4
    bricks = (4, 4, 4)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=bricks, dtype="f32", layout="cell8")
    fld.set_global(F)
    del F
    seeds = torch.from_numpy(inputs.uniform_seeds(g, n_seeds, rank_seed(1, rank))).to(dev)
    stream = torch.cuda.current_stream(dev)
    undivided = api.Tracer(ctx, fld, capacity=n_seeds, dt=dt, max_steps=max_steps)

    def run_undivided():
        undivided.upload_seeds(seeds)
        undivided.trace()

    owner = pod.partition_bricks(bricks, ranks)
    engines = [pod.GpuEngine(api.Tracer(ctx, fld, capacity=n_seeds, dt=dt, max_steps=max_steps), owner, r, ranks)
               for r in range(ranks)]
    rounds = [0]

    def run_pod_once():
        for e in engines:
            e.tr.upload_seeds(seeds)
        rounds[0] = pod.LocalTransport.trace_local(engines)

    ms_u = _cuda_ms(run_undivided, args.steps, args.warmup, stream)
    ms_p = _cuda_ms(run_pod_once, args.steps, args.warmup, stream)
    steps = undivided.total_steps()
    got = engines[0].tr.get_lines()
    ref = undivided.get_lines()
    torch.cuda.synchronize(dev)
    same = bool(torch.equal(got.offsets, ref.offsets) and torch.equal(got.vertices, ref.vertices))
    out = {"metric": METRIC + " (partition over data, 4 ranks emulated on one GPU)", "value": steps / (ms_p / 1e3),
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_p,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "partition over data: 512^3 FP32 turbulence (seed 1), 64 bricks (4x4x4) over 4 "
                                  "ranks emulated as tracers on one GPU, CELL8, 262144 seeds, max 1000 steps, RK4 "
                                  "h=0.5 cell", "ranks": ranks, "exchange_rounds": rounds[0]},
           "particle_steps_per_step": steps, "undivided": {"value": steps / (ms_u / 1e3), "ms_per_step": ms_u},
           "merged_lines_equal_undivided": same}
    print(json.dumps(out))


def run_serve(args, rank, world, local):
    """The serving workload on its own, with the autotuner's schedule (config 5)."""
    import torch
    from paper_2606_02627_gb300 import api
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    ctx = api.Context(local)
    st = serve_workload(ctx, dev, args.requests, args.h, rank=rank, tune=True)
    out = {"metric": "p99 request latency (serving)", "value": st["p99_ms"], "unit": "ms", "n_gpus": 1,
           "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+bf16", "data": "synthetic",
           "config": {"workload": SERVE_WORKLOAD + f" ({args.requests} requests, {st['rate_per_s']:.1f}/s)",
                      "rounds_per_launch": st["rounds_per_launch"], "slab_pool_bytes": st["slab_pool_bytes"],
                      "schedule": st["schedule"]},
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
           "particle_steps_per_s": st["particle_steps_per_s"], "particle_steps": st["particle_steps"],
           "capacity": st["capacity"], "queue_ms_p99": st["queue_ms_p99"]}
    print(json.dumps(out))


def run_plain(args, rank, world, local):
    """The plain method on one brick: a 64^3 FP32 field of solid-body rotation and of ABC flow on [0, 2pi]^3,
    1024 seeds uniform in the interior (seed 0), RK4 with h = 0.25 cell, max 500 steps, stop on exit or
    |v| < 1e-6; the persistent kernel on CELL8 records and the plain per-seed kernel on the float3 array.
    One step = seed upload + trace + CSR compaction (the field stays resident).  Latency-bound: 1024 lines
    on 152 SMs."""
    import torch
    from paper_2606_02627_gb300 import api, inputs
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    ctx = api.Context(local)
    g = inputs.cube_grid(64)
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 1024, 0, lo_cells=1.0)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for which in ("rotation", "abc"):
        F = inputs.rotation_field(g) if which == "rotation" else inputs.abc_field(g)
        Fd = torch.from_numpy(F).to(dev)
        sp = torch.tensor(g.spacing, device=dev, dtype=torch.float32)
        dt = 0.25 / float((Fd / sp).norm(dim=-1).max())
        for kernel, layout in (("persistent", "cell8"), ("per_seed", "global")):
            fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(1, 1, 1), dtype="f32", layout=layout)
            fld.set_global(Fd, stream=stream)
            tr = api.Tracer(ctx, fld, capacity=1024, dt=dt, max_steps=500, kernel=kernel)
            nl = tr.capacity
            off = torch.empty(nl + 1, dtype=torch.int64, device=dev)
            vert = torch.empty((nl * 501, 3), dtype=torch.float32, device=dev)

            def one():
                tr.upload_seeds(seeds, stream=stream)
                tr.trace(stream=stream)
                api.call("sg_tracer_get_lines", tr.h, None, None, api._ptr(off), api._ptr(vert), None, None, None,
                         api._stream(stream))
            for _ in range(args.warmup):
                one()
            stream.synchronize()
            steps = tr.total_steps(stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                one()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            res[f"{which}_{kernel}"] = {"value": steps / (ms / 1e3), "ms_per_step": ms, "particle_steps": steps}
            del tr, fld
    out = {"metric": "RK4 particle-steps/s (plain method, one brick)", "value": res["abc_persistent"]["value"],
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res["abc_persistent"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "plain method: 64^3 FP32 rotation / ABC flow on [0,2pi]^3, 1 brick, 1024 seeds "
                                  "(seed 0), RK4 h=0.25 cell, max 500 steps"},
           "variants": res}
    print(json.dumps(out))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.config == "plain":
        return run_plain(args, rank, world, local)
    if args.config in ("streak", "umesh") and args.dtype != "f32":
        raise SystemExit(f"--config {args.config} stores its field in FP32 only (--dtype f32)")
    if args.config == "streak":
        return run_streak(args, rank, world, local)
    if args.config == "serve":
        return run_serve(args, rank, world, local)
    if args.config == "umesh":
        return run_umesh(args, rank, world, local)
    if args.config == "bidir":
        return run_bidir(args, rank, world, local)
    if args.config == "path":
        return run_path(args, rank, world, local)
    if args.config == "pod":
        return run_pod(args, rank, world, local)
    import numpy as np
    import torch

    from paper_2606_02627_gb300 import inputs

    n = args.n
    grid = inputs.cube_grid(n)
    config = {"workload": f"steady streamlines, {n}^3 FP32 vec3 synthetic turbulence (256 modes, seed 1), "
                          f"4x4x4 bricks + 1-cell ghost, {args.seeds} seeds, RK4 h={args.h} cell, "
                          f"max {args.max_steps} steps",
              "field": f"{n}^3", "bricks": "4x4x4", "seeds_per_gpu": args.seeds, "max_steps": args.max_steps,
              "h_cells": args.h, "field_storage": args.dtype, "layout": args.layout,
              "l2": "inputs larger than L2 (field 1.6 GB; cell records 13.5 GB FP32, 9 GB 8-byte formats; "
                    "slabs 24 GB)",
              "parallelism": f"replicas x{world} (seeds per rank, field replicated)"}

    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm is the FP64 oracle on the host cores, on a bounded prefix of the seeds
        import oracle
        modes = inputs.turbulence_modes(1)
        F = inputs.turbulence_field(grid, modes, device="cuda" if torch.cuda.is_available() else None)
        F_host = F.cpu().numpy()
        del F
        dt = args.h / oracle.max_speed(F_host, grid.spacing)
        seeds = inputs.uniform_seeds(grid, args.seeds, 1)
        rates = []
        info = None
        for it in range(args.warmup + args.steps):
            # the first step sizes the prefix; every step traces the same seeds
            rate, cores, ns, steps, secs = cpu_oracle_rate(F_host, grid, seeds, dt, args.max_steps,
                                                           args.cpu_seconds / 2, n_seeds=info[1] if info else None)
            if it >= args.warmup:
                rates.append(rate)
            info = (cores, ns, steps, secs)
        v = statistics.median(rates)
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
               "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64", "data": "synthetic", "config": config,
               "cpu_baseline": {"value": v, "unit": UNIT, "cores": info[0], "kind": "oracle",
                                "sample": f"first {info[1]} of {args.seeds} seeds per step ({info[2]} particle-steps, "
                                          f"{info[3]:.1f} s)"},
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    from paper_2606_02627_gb300 import api
    from paper_2606_02627_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.Stream(device=dev)
    ctx = api.Context(local)

    modes = inputs.turbulence_modes(1)
    with torch.cuda.stream(stream):
        F = inputs.turbulence_field(grid, modes, device=dev)
    stream.synchronize()
    sched = {}
    if args.schedule:
        vals = [int(x) for x in args.schedule.split(",")]
        sched = dict(block_size=vals[0], blocks_per_sm=vals[1], steps_per_round=vals[2])
        if len(vals) > 3:
            sched["drain_steps"] = vals[3]

    seeds_np = inputs.uniform_seeds(grid, args.seeds, rank_seed(1, rank))
    seeds_dev = torch.from_numpy(seeds_np).to(dev)
    seeds_pin = torch.from_numpy(seeds_np).pin_memory() if not args.no_e2e else None

    def make(dtype, layout, kernel, bricks=(4, 4, 4), extra=None):
        fld = api.Field(ctx, grid.dims, grid.origin, grid.spacing,
                        bricks=(1, 1, 1) if layout == "global" else tuple(bricks), dtype=dtype, layout=layout)
        fld.set_global(F, stream=stream)
        kw = dict(sched) if kernel in ("persistent", "lockstep") else {}
        kw.update(extra or {})
        tr = api.Tracer(ctx, fld, capacity=args.seeds, dt=dt, max_steps=args.max_steps, kernel=kernel, **kw)
        return fld, tr

    # dt from the FP32 field's largest speed: every step is at most h cells
    probe = api.Field(ctx, grid.dims, grid.origin, grid.spacing, bricks=(4, 4, 4), dtype="f32")
    probe.set_global(F, stream=stream)
    vref = probe.max_speed(stream=stream)
    dt = args.h / vref
    del probe

    def one_step(fld, tr, out_off, out_vert, out_st, seeds):
        fld.set_global(F, stream=stream)                     # a1: bricks, ghosts, encode
        tr.upload_seeds(seeds, stream=stream)               # a2: seeds -> per-brick queues
        if args.host_loop:
            tr.trace_timed(stream=stream)                   # a3-a7, rounds driven from the host
        else:
            tr.trace(stream=stream)                         # a3-a7: rounds of the persistent kernel (graph)
        if out_off is not None and not out_off.is_cuda:
            # a8 into page-locked host memory: the copy overlaps the next step
            api.call("sg_tracer_get_lines_overlapped", tr.h, None, None, api._ptr(out_off), api._ptr(out_vert),
                     api._ptr(out_st), None, api._stream(stream))
        else:
            api.call("sg_tracer_get_lines", tr.h, None, None, api._ptr(out_off), api._ptr(out_vert),
                     api._ptr(out_st), None, None, api._stream(stream))    # a8: CSR

    def timed(fld, tr, warmup, steps, seeds, host_out=False):
        nl, nv = None, None
        # size the outputs from one untimed run
        one_step(fld, tr, None, None, None, seeds_dev)
        nl, nv = tr.sizes(stream=stream)
        tot = tr.total_steps(stream=stream)
        kw = dict(pin_memory=True) if host_out else dict(device=dev)
        off = torch.empty(nl + 1, dtype=torch.int64, **kw)
        vert = torch.empty((max(nv, 1), 3), dtype=torch.float32, **kw)
        st = torch.empty(max(nl, 1), dtype=torch.uint8, **kw)
        for _ in range(warmup):
            one_step(fld, tr, off, vert, st, seeds)
        if host_out:
            tr.wait_lines(stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            one_step(fld, tr, off, vert, st, seeds)
        if host_out:
            tr.wait_lines(stream)                           # the last step's lines are on the host
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        ms, tot_all = reduce_over_ranks(ms, tot, dist, dev)
        ok = tr.check(stream=stream)
        bytes_out = off.numel() * 8 + nv * 12 + nl
        if host_out:
            # the copy rate into the step's own page-locked output (its first 2 GiB), after the timed region:
            # sets a slow host buffer apart from a slow pipeline
            n = min(vert.numel(), 1 << 29)
            src = torch.empty(n, dtype=torch.float32, device=dev)
            best = None
            for _ in range(3):
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                with torch.cuda.stream(stream):
                    vert.view(-1)[:n].copy_(src, non_blocking=True)
                c1.record(stream)
                c1.synchronize()
                best = c0.elapsed_time(c1) if best is None else min(best, c0.elapsed_time(c1))
            timed.out_buffer_gbs = n * 4 / (best / 1e3) / 1e9
            del src
        return ms, tot, tot_all, bytes_out

    results = {}
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass

    # headline: the chosen storage type and persistent kernel, on the structure and schedule the autotuner
    # picks for this workload (successive halving over layouts, brick shapes, brick windows and schedules on
    # growing prefixes of the same seeds, up to all of them)
    tuned = None
    head_bricks, head_extra, head_layout = (4, 4, 4), {}, args.layout
    if not args.no_tune and not args.schedule and args.kernel == "persistent" and not args.once:
        from paper_2606_02627_gb300 import autotune
        t0 = time.time()
        # the workload fixes the decomposition (4x4x4 bricks): layouts, brick windows and schedules are tuned
        choice = autotune.tune_structure(ctx, F, grid, args.dtype, seeds_dev, dt, args.max_steps, first=1 << 16,
                                         structs=autotune.structures(64, bricks=((4, 4, 4),)),
                                         cache=os.path.join(tempfile.gettempdir(), f"streamgb_tune_{os.getpid()}.json"),
                                         stream=stream)
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        head_layout, head_bricks = choice["layout"], tuple(choice["bricks"])
        head_extra = dict(choice["schedule"], brick_window=choice["brick_window"])
        tuned = dict(choice, seconds=round(time.time() - t0, 1))
        config.update(layout=head_layout, bricks="x".join(map(str, head_bricks)))
    config["schedule"] = tuned or {"schedule": "library default" if not args.schedule else sched}
    fld, tr = make(args.dtype, head_layout, args.kernel, head_bricks, head_extra)
    if args.once:
        # one whole step: field store, seeds, rounds, and the CSR gathered into device buffers
        one_step(fld, tr, None, None, None, seeds_dev)
        nl, nv = tr.sizes(stream=stream)
        o_off = torch.empty(nl + 1, dtype=torch.int64, device=dev)
        o_vert = torch.empty((max(nv, 1), 3), dtype=torch.float32, device=dev)
        o_st = torch.empty(max(nl, 1), dtype=torch.uint8, device=dev)
        api.call("sg_tracer_get_lines", tr.h, None, None, api._ptr(o_off), api._ptr(o_vert), api._ptr(o_st), None,
                 None, api._stream(stream))
        stream.synchronize()
        print(json.dumps({"once": True, "particle_steps": tr.total_steps(stream=stream),
                          "rounds": tr.check(stream=stream), "dtype": args.dtype, "layout": args.layout,
                          "n": n, "seeds": args.seeds, "max_steps": args.max_steps}))
        return
    with Clocks(uuid) as clk:
        ms, tot, tot_all, _ = timed(fld, tr, args.warmup, args.steps, seeds_dev)
    clocks = clk.summary()
    value = tot_all / (ms / 1e3)
    results["headline"] = (ms, tot)

    # roofline of the dominant kernel: round kernel time by CUDA events (host-driven rounds)
    tr.upload_seeds(seeds_dev, stream=stream)
    fld.set_global(F, stream=stream)
    kms, launches = tr.trace_timed(stream=stream)
    ksteps = tr.total_steps(stream=stream)
    hbm, peak_kind = peaks()
    bps = GATHER_BYTES[args.dtype]
    k_rate = ksteps / (kms / 1e3)                       # particle-steps/s of the advection kernel alone
    tag = "async" if args.kernel == "persistent" and head_layout == "cell8" else "lockstep"
    cnt = counters(args.dtype, tag)
    tps = cnt.get("dram_bytes_per_particle_step")
    tips = cnt.get("thread_inst_per_particle_step")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    gather = ksteps * bps / (kms / 1e3) / 1e9
    roofline = {"bound": "issue", "achieved": None, "peak": None, "unit": "G thread-instructions/s", "frac": None,
                "traffic": (tps * ksteps / launches) if tps else None,
                "kernel": ("round_async_kernel (persistent advection, decoupled lanes)"
                           if tag == "async" else "round_kernel (persistent advection, lanes in lockstep)"),
                "peak_source": f"{sm_count} SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz (median SM clock "
                               "under load in this run): one warp instruction per scheduler per cycle",
                "model": "thread instructions per particle-step (ncu smsp__thread_inst_executed.sum over every "
                         "advection launch of one trace, committed in profiles/) x the kernel's particle-steps/s",
                "kernel_ms_per_launch": kms / launches, "launches": launches,
                "particle_steps_per_launch": ksteps / launches, "kernel_particle_steps_per_s": k_rate,
                "thread_inst_per_particle_step": tips,
                "threads_per_warp_inst": cnt.get("threads_per_warp_inst"),
                "gather_model": {"achieved": gather, "peak": hbm, "unit": "GB/s", "frac": gather / hbm,
                                 "peak_source": f"{peak_kind} hbm_gbs",
                                 "model": f"4 samples x 8 corners x 3 comps x elem + 12 B vertex = {bps} B per "
                                          "particle-step (hits in the lane's record slot, L1 and L2 counted at "
                                          "HBM price)"},
                "dram": ({"bytes_per_particle_step": tps, "achieved": tps * k_rate / 1e9, "peak": hbm,
                          "unit": "GB/s", "frac": tps * k_rate / 1e9 / hbm, "peak_source": f"{peak_kind} hbm_gbs"}
                         if tps else None)}
    if tips:
        a, pk, fr = issue_roofline(k_rate, tips, sm_count, sm_mhz)
        roofline.update(achieved=a, peak=pk, frac=fr)

    # e2e through the C ABI: seeds from pinned host, CSR lines to pinned host (copy overlapping the next
    # step), inside the timed region
    e2e = None
    if not args.no_e2e:
        ems, _, etot_all, d2h = timed(fld, tr, 2, max(1, args.steps), seeds_pin, host_out=True)
        e2e = {"value": etot_all / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(seeds_pin.numel() * 4),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ems}
        # the host link it runs on: one 2 GiB page-locked copy each way (the step's D2H copy overlaps the next
        # step's trace, so the step takes about max(trace, D2H copy) plus the pipeline's fill and drain)
        e2e.update(copy_rates(dev))
        e2e["d2h_ms_per_step"] = d2h / (e2e["d2h_gbs"] * 1e9) * 1e3
        e2e["d2h_gbs_into_output"] = getattr(timed, "out_buffer_gbs", None)
    del tr, fld
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants:
        runs = [(f"{d}_persistent", d, args.layout, "persistent") for d in ("fx21", "f16", "bf16", "f32")
                if d != args.dtype]
        other = "lockstep" if args.kernel == "persistent" else "persistent"
        runs.append((f"{args.dtype}_{other}", args.dtype, args.layout, other))
        runs.append(("f32_per_seed", "f32", "global", "per_seed"))
        if args.per_step:
            runs.append(("f32_per_step", "f32", args.layout, "per_step"))
        for name, dtp, lay, ker in runs:
            f2, t2 = make(dtp, lay, ker)
            vms, vtot, vtot_all, _ = timed(f2, t2, 1, 2, seeds_dev)
            variants[name] = {"value": vtot_all / (vms / 1e3), "ms_per_step": vms, "particle_steps": vtot,
                              "field_storage": dtp, "kernel": ker}
            del t2, f2
            torch.cuda.empty_cache()
        variants[f"{args.dtype}_{args.kernel}"] = {"value": value, "ms_per_step": ms, "particle_steps": tot,
                                                   "field_storage": args.dtype, "kernel": args.kernel}

    serve = None
    if args.serve_requests > 0:
        # continuous batching of interactive seed placement (config 5's recipe, a shorter request stream):
        # p50 / p99 request latency beside the throughput
        serve = serve_workload(ctx, dev, args.serve_requests, args.h, rank=rank, tune=False)
        serve["workload"] = SERVE_WORKLOAD + f" ({args.serve_requests} requests)"

    cpu = None
    if rank == 0:
        F_host = F.cpu().numpy()
        rate, cores, ns, steps, secs = cpu_oracle_rate(F_host, grid, seeds_np, dt, args.max_steps, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {ns} of {args.seeds} seeds of the same workload on the FP32 field "
                         f"({steps} particle-steps in {secs:.1f} s)"}
        # the same oracle on one core, over a shorter prefix
        rate1, _, ns1, steps1, secs1 = cpu_oracle_rate(F_host, grid, seeds_np, dt, args.max_steps,
                                                       args.cpu_seconds / 4, nthreads=1)
        cpu["one_core"] = {"value": rate1, "unit": UNIT,
                           "sample": f"first {ns1} seeds ({steps1} particle-steps in {secs1:.1f} s)"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.dtype, "data": "synthetic", "config": config,
               "particle_steps_per_step": tot_all, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "serving": serve, "gpu_launches": None, "clocks": clocks, "variants": variants}
        # kernels of ours per timed step: set_global (2-3), upload (1), prepare (1), bin (4) + rounds x (1 + 4),
        # park_rest (1), scan (3), gather (1)
        out["gpu_launches"] = int(args.steps * (3 + 1 + 1 + 4 + launches * 5 + 1 + 3 + 1))
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
