"""Path lines (every seed released once at time 0, followed through the
time-dependent field) on the GPU, against the FP64 oracle.

Time slices are streamed from page-locked host memory into three resident
slots on a side stream while the tracer steps (the streakline machinery);
each step samples the field linear in time between the slices of its stage
times.  Checked: every vertex within 1e-3 cells of the oracle's path line,
statuses and lengths equal (up to boundary ties), the steady case against the
streamline tracer, max_steps, OUT seeds and the missing-slice error.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs
from tests.helpers import compare_lines

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    return api.Context(0)


def run_pathlines(ctx, g, slices, sdt, seeds, dt, max_steps, dtype="f32", layout="linear", bricks=(2, 2, 2),
                  step_chunk=1):
    from paper_2606_02627_gb300 import api
    n_slices = len(slices)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=bricks, dtype=dtype, layout=layout, n_slots=3,
                    slice_dt=sdt)
    pinned = [torch.from_numpy(np.ascontiguousarray(slices[s])).pin_memory() for s in range(n_slices)]
    side = torch.cuda.Stream()
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=max_steps, mode="pathline")
    fld.stream_slice(0, pinned[0], stream=side)
    fld.stream_slice(1, pinned[1], stream=side)
    tr.upload_seeds(torch.from_numpy(seeds).cuda())
    j = 0
    while j < max_steps:
        # step j+1 spans times j dt .. (j+1) dt: with sdt == dt it needs slices j, j+1
        if j + 2 < n_slices:
            fld.stream_slice(j + 2, pinned[j + 2], stream=side)
        active = tr.step(1)
        j += 1
        if not active:
            break
    lines = tr.get_lines()
    torch.cuda.synchronize()
    return tr, lines


@pytest.mark.parametrize("dtype,layout", [("f32", "linear"), ("f32", "cell8")])
def test_pathlines_match_oracle(ctx, dtype, layout):
    n = 41
    g = inputs.cube_grid(n)
    modes = inputs.turbulence_modes(5, n_modes=64, kmax=2)
    n_slices = 26
    slices = np.stack([inputs.turbulence_field(g, modes, time_slice=s, n_slices=n_slices).numpy()
                       for s in range(n_slices)])
    vref = max(oracle.max_speed(slices[s], g.spacing) for s in range(n_slices))
    dt = 0.5 / vref
    sdt = dt
    seeds = inputs.uniform_seeds(g, 700, 5)
    seeds[:3] = np.float32(-5.0)                 # OUT
    steps = n_slices - 1
    ref = oracle.trace_pathlines(slices, g.origin, g.spacing, sdt, seeds, dt, steps, eps=1e-6)
    tr, lines = run_pathlines(ctx, g, slices, sdt, seeds, dt, steps, dtype, layout)
    st = compare_lines(lines, g, ref, tol=1e-3)
    assert st["vertices"] > 700 * 10
    assert tr.total_steps() == int(np.maximum(ref.length.astype(np.int64) - 1, 0).sum())


def test_steady_pathlines_are_streamlines(ctx):
    from paper_2606_02627_gb300 import api
    n = 33
    g = inputs.cube_grid(n)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(6, n_modes=48, kmax=2)).numpy()
    slices = np.stack([F] * 40)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    seeds = inputs.uniform_seeds(g, 400, 6)
    _, pl = run_pathlines(ctx, g, slices, dt, seeds, dt, 30)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(2, 2, 2))
    fld.set_global(torch.from_numpy(F).cuda())
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=30)
    tr.upload_seeds(torch.from_numpy(seeds).cuda())
    tr.trace()
    sl = tr.get_lines()
    assert torch.equal(pl.offsets, sl.offsets)
    assert torch.equal(pl.status & 0x7F, sl.status & 0x7F)
    d = (pl.vertices - sl.vertices).abs().max().item()
    assert d < 1e-4 * max(g.spacing)


def test_pathline_max_steps_and_missing_slice(ctx):
    from paper_2606_02627_gb300 import api
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    F = inputs.uniform_field(g, (0.25, 0.0, 0.0))
    slices = np.stack([F] * 6)
    seeds = np.array([[1.0, 4.0, 4.0], [-1.0, 4.0, 4.0]], dtype=np.float32)
    for ms in (0, 1, 3):
        _, lines = run_pathlines(ctx, g, slices, 1.0, seeds, 1.0, ms)
        assert lines.lengths().cpu().tolist() == [ms + 1, 0]
        assert (lines.status.cpu().numpy() & 0x7F).tolist() == [oracle.MAXSTEPS, oracle.OUT]
        assert np.allclose(lines.vertices.cpu().numpy()[:, 0], 1.0 + 0.25 * np.arange(ms + 1))
    # a step whose time slices are not resident is refused
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(1, 1, 1), n_slots=3, slice_dt=1.0)
    fld.stream_slice(0, torch.from_numpy(F).pin_memory())
    tr = api.Tracer(ctx, fld, capacity=2, dt=1.0, max_steps=5, mode="pathline")
    tr.upload_seeds(torch.from_numpy(seeds).cuda())
    with pytest.raises(api.L.StreamGBError):
        tr.step(1)
    with pytest.raises(api.L.StreamGBError):
        tr.trace()
