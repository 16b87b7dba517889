"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

* 512^3 turbulence (seed 1), 4x4x4 bricks, 1M uniform seeds, h = 0.5 cell,
  max 2000 steps, FX21 + CELL8 storage and FP32 + CELL8, default schedule:
  2048 sampled lines against the FP64 oracle on the FP32 field, plus
  properties that hold for every line (status set, lengths within the cap,
  vertices inside the domain, total steps = sum of lengths - 1).
* The same 512^3 FP32 workload under the schedules the autotuner picks for
  the benchmark's headline (256 x 4 CTAs per SM and 512 steps per round; 128
  x 6 and 128 steps with no drain limit): the same lines, bit for bit, as the
  default schedule (whose lines are checked against the oracle above).
* 1024^3 turbulence (seed 2), 4M seeds, max 1000 steps, FP32 / FX21 / BF16 /
  FP16 storage: vertex error on the first 10k seeds against the FP64 oracle on
  the FP32 field (max and p99 reported; the 1e-3 FP32 bound and the 5e-2
  precision bound asserted on every vertex for FP32 and FX21, at the 99th
  percentile for BF16 and FP16).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs
from tests.helpers import compare_lines

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    return api.Context(0)


class Sub:
    """A subset of CSR lines as an object compare_lines accepts."""

    def __init__(self, lines, idx):
        dev = lines.offsets.device
        ii = torch.as_tensor(idx, device=dev)
        start = lines.offsets[ii]
        lens = lines.offsets[ii + 1] - start
        owner = torch.repeat_interleave(torch.arange(len(idx), device=dev), lens)
        new_off = torch.zeros(len(idx) + 1, dtype=torch.int64, device=dev)
        new_off[1:] = torch.cumsum(lens, 0)
        pos = torch.arange(int(new_off[-1]), device=dev) - new_off[:-1][owner] + start[owner]
        self.offsets = new_off.cpu()
        self.vertices = lines.vertices[pos].cpu()
        self.status = lines.status[ii].cpu()
        self.margin = lines.margin[ii].cpu()


def trace_full(ctx, g, F, seeds, dt, max_steps, dtype, layout="cell8", **sched):
    from paper_2606_02627_gb300 import api
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4), dtype=dtype, layout=layout)
    fld.set_global(F)
    tr = api.Tracer(ctx, fld, capacity=seeds.shape[0], dt=dt, max_steps=max_steps, **sched)
    tr.upload_seeds(seeds)
    tr.trace()
    tr.check()
    lines = tr.get_lines()
    steps = tr.total_steps()
    torch.cuda.synchronize()
    tr.close()
    fld.close()
    return lines, steps


def check_properties(lines, g, n, max_steps, steps):
    lens = lines.lengths().cpu().numpy()
    st = lines.status.cpu().numpy() & 0x7F
    assert len(lens) == n
    assert set(np.unique(st)) <= {1, 2, 3, 4, 5}
    assert lens.max() <= max_steps + 1 and lens.min() >= 0
    assert (lens[st == 1] == max_steps + 1).all()                    # MAXSTEPS lines are full
    assert int(np.maximum(lens - 1, 0).sum()) == steps
    v = lines.vertices
    lo = torch.tensor(g.origin, device=v.device) - 1e-4
    hi = torch.tensor([g.origin[a] + g.spacing[a] * (g.dims[a] - 1) for a in range(3)], device=v.device) + 1e-4
    assert bool(((v >= lo) & (v <= hi)).all())


def test_512_bench_configuration_sampled_lines(ctx):
    g = inputs.cube_grid(512)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1), device="cuda")
    seeds_np = inputs.uniform_seeds(g, 1 << 20, 1)
    seeds = torch.from_numpy(seeds_np).cuda()
    from paper_2606_02627_gb300 import api
    probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4))
    probe.set_global(F)
    dt = 0.5 / probe.max_speed()
    probe.close()
    F_host = F.cpu().numpy()
    idx = np.sort(np.random.default_rng(0).choice(1 << 20, 2048, replace=False))
    ref = oracle.trace_streamlines(F_host, g.origin, g.spacing, seeds_np[idx], dt, 2000, eps=1e-6,
                                   nthreads=oracle.default_threads())
    for dtype, tol in (("fx21", 5e-2), ("f32", 5e-3)):
        lines, steps = trace_full(ctx, g, F, seeds, dt, 2000, dtype)
        check_properties(lines, g, 1 << 20, 2000, steps)
        sub = Sub(lines, idx)
        st = compare_lines(sub, g, ref, tol=tol, tie_cells=max(tol, 1e-3))
        print(f"512^3 {dtype}: {steps} particle-steps; sampled max err {st['max_err']:.2e} p99 {st['p99']:.2e} "
              f"ties {st['ties']}")
        if dtype == "f32":
            # the FP32 bound is stated after 1000 steps: the first 1001 vertices of every sampled line
            off = sub.offsets.numpy()
            v = (sub.vertices.numpy().astype(np.float64) - np.array(g.origin)) / np.array(g.spacing)
            e1000 = max(float(np.abs(v[off[i]:off[i] + k] - ref.line(i)[:k]).max())
                        for i in range(len(idx)) for k in [min(off[i + 1] - off[i], ref.length[i], 1001)] if k)
            print(f"512^3 f32: max err over the first 1000 steps {e1000:.2e}")
            assert e1000 <= 1e-3


def test_512_tuned_schedules_same_bits(ctx):
    g = inputs.cube_grid(512)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1), device="cuda")
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 1 << 20, 1)).cuda()
    from paper_2606_02627_gb300 import api
    probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4))
    probe.set_global(F)
    dt = 0.5 / probe.max_speed()
    probe.close()
    base, steps = trace_full(ctx, g, F, seeds, dt, 2000, "f32")
    for sched in (dict(block_size=256, blocks_per_sm=4, steps_per_round=512),
                  dict(block_size=128, blocks_per_sm=6, steps_per_round=128, drain_steps=-1)):
        lines, st = trace_full(ctx, g, F, seeds, dt, 2000, "f32", **sched)
        assert st == steps
        assert torch.equal(lines.offsets, base.offsets)
        assert torch.equal(lines.status, base.status)
        assert torch.equal(lines.vertices, base.vertices), sched
        del lines
        torch.cuda.empty_cache()


def test_1024_precision_forms_error_on_10k_seeds(ctx):
    g = inputs.cube_grid(1024)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(2), device="cuda")
    seeds_np = inputs.uniform_seeds(g, 4 << 20, 2)
    seeds = torch.from_numpy(seeds_np).cuda()
    from paper_2606_02627_gb300 import api
    probe = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(4, 4, 4))
    probe.set_global(F)
    dt = 0.5 / probe.max_speed()
    probe.close()
    F_host = F.cpu().numpy()
    ref = oracle.trace_streamlines(F_host, g.origin, g.spacing, seeds_np[:10000], dt, 1000, eps=1e-6,
                                   nthreads=oracle.default_threads())
    idx = np.arange(10000)
    report = {}
    for dtype, layout in (("f32", "linear"), ("fx21", "cell8"), ("bf16", "cell8"), ("f16", "cell8")):
        lines, steps = trace_full(ctx, g, F, seeds, dt, 1000, dtype, layout)
        check_properties(lines, g, 4 << 20, 1000, steps)
        st = compare_lines(Sub(lines, idx), g, ref, tol=1e9, tie_cells=0.5)
        report[dtype] = (st["max_err"], st["p99"])
        print(f"1024^3 {dtype}/{layout}: max err {st['max_err']:.3e} p99 {st['p99']:.3e} cells")
        del lines
        torch.cuda.empty_cache()
    assert report["f32"][0] <= 1e-3
    assert report["fx21"][0] <= 5e-2
    # BF16 and FP16 meet the stated 5e-2-cell bound at the 99th percentile of
    # the vertices (their largest errors are reported, not bounded)
    assert report["bf16"][1] <= 5e-2
    assert report["f16"][1] <= 5e-2
