"""The allocation-free compaction entry point (sg_lines_compact_static).

Some callers cannot allocate device memory while they hand work to this
library: an in-situ simulation that keeps all of HBM in its own pool, or a
loop that cannot take the synchronisation cudaMalloc/cudaFree may cause.
For them sg_lines_compact_static keeps its scan scratch in a fixed array
inside the library.  This test calls it through the C ABI and checks its
output against sg_tracer_get_lines on the same lines, twice in a row (the
second call must not see anything left over from the first).  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    return api.Context(0)


def traced_lines(ctx, n_seeds, max_steps, seed):
    from paper_2606_02627_gb300 import api
    g = inputs.cube_grid(48)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(seed, n_modes=64, kmax=3)).numpy()
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(2, 3, 2))
    fld.set_global(torch.from_numpy(F).cuda())
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    tr = api.Tracer(ctx, fld, capacity=n_seeds, dt=dt, max_steps=max_steps)
    tr.upload_seeds(torch.from_numpy(inputs.uniform_seeds(g, n_seeds, seed)).cuda())
    tr.trace()
    lines = tr.get_lines()
    torch.cuda.synchronize()
    return lines


def slab_of(lines, W):
    """Rebuilds per-line slabs [n][W][3] and lengths from CSR lines (torch ops)."""
    off = lines.offsets
    n = off.numel() - 1
    lens = (off[1:] - off[:-1])
    slab = torch.full((n, W, 3), float("nan"), device=off.device)
    line_of = torch.repeat_interleave(torch.arange(n, device=off.device), lens)
    pos = torch.arange(int(off[-1]), device=off.device) - off[:-1][line_of]
    slab[line_of, pos] = lines.vertices
    return slab.contiguous(), lens.to(torch.int32).contiguous()


def compact_static(slab, lens, W, offsets, vertices):
    from paper_2606_02627_gb300 import _lib
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.call("sg_lines_compact_static", ctypes.c_void_p(slab.data_ptr()), W, ctypes.c_void_p(lens.data_ptr()),
              lens.numel(), ctypes.c_void_p(offsets.data_ptr()),
              ctypes.c_void_p(vertices.data_ptr()) if vertices is not None else None, s)


def test_static_compaction_matches_get_lines_twice(ctx):
    W = 301
    for n_seeds, seed in ((5000, 3), (1234, 11)):        # two calls in a row, different sizes
        lines = traced_lines(ctx, n_seeds, W - 1, seed)
        slab, lens = slab_of(lines, W)
        off = torch.full((n_seeds + 1,), -7, dtype=torch.int64, device="cuda")
        vert = torch.full_like(lines.vertices, float("nan"))
        compact_static(slab, lens, W, off, vert)
        torch.cuda.synchronize()
        assert torch.equal(off, lines.offsets)
        assert torch.equal(vert, lines.vertices)


def test_static_compaction_to_pinned_host_and_offsets_only(ctx):
    W = 201
    lines = traced_lines(ctx, 3000, W - 1, 5)
    slab, lens = slab_of(lines, W)
    off_h = torch.empty(3001, dtype=torch.int64).pin_memory()
    vert_h = torch.empty(tuple(lines.vertices.shape), dtype=torch.float32).pin_memory()
    compact_static(slab, lens, W, off_h, vert_h)
    torch.cuda.synchronize()
    assert torch.equal(off_h, lines.offsets.cpu())
    assert torch.equal(vert_h, lines.vertices.cpu())
    off2 = torch.zeros(3001, dtype=torch.int64, device="cuda")
    compact_static(slab, lens, W, off2, None)
    torch.cuda.synchronize()
    assert torch.equal(off2, lines.offsets)


def test_static_compaction_rejects_oversize():
    from paper_2606_02627_gb300 import _lib
    L = _lib.lib()
    rc = L.sg_lines_compact_static(None, 10, None, (4096 * 4096) + 1, ctypes.c_void_p(8), None, None)
    assert rc == _lib.SG_ERR_INVALID_ARG
    assert "exceeds the limit" in _lib.last_error()
