"""Autotuner of the persistent kernel (successive halving over structures and
schedules): candidate grids on the CPU; on the GPU, the tuners return one of
their candidates and cache it per problem shape, and neither a schedule, a
layout, a brick shape nor a brick window changes a bit of the lines (they
decide only which lane advances which particle when, and where its samples
are stored).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs


def test_candidates_are_valid_schedules():
    from paper_2606_02627_gb300 import autotune
    cands = autotune.candidates()
    assert len(cands) == len(set(cands)) > 20
    for block, bps, spr, drain in cands:
        assert block % 32 == 0 and 32 <= block <= 256
        assert 256 <= block * bps <= 1024
        assert spr > 0 and drain in (0, -1)
    assert all(c[0] * c[1] <= 512 for c in autotune.candidates(max_threads_per_sm=512))
    s = autotune.schedule_of((128, 6, 256, -1))
    assert s == dict(block_size=128, blocks_per_sm=6, steps_per_round=256, drain_steps=-1)


def test_structures_cover_layouts_bricks_and_windows():
    from paper_2606_02627_gb300 import autotune
    st = autotune.structures(64)
    assert len(st) == len(set(st))
    assert {s[0] for s in st} == {"cell8", "tiled4", "linear"}
    assert {s[1] for s in st} == {(2, 2, 2), (4, 4, 4), (8, 8, 8)}
    assert {s[2] for s in st} == {0, 8, 32}                # every brick, an eighth and half of 64
    assert all(s[2] == 0 or s[0] == "cell8" for s in st)
    assert autotune.structures(64, windows=(3,))[-1] == ("cell8", (4, 4, 4), 3)


@pytest.fixture(scope="module")
def small():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    ctx = api.Context(0)
    g = inputs.cube_grid(49)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(21, n_modes=48, kmax=3)).numpy()
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 6000, 21)).cuda()
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    return ctx, g, F, seeds, dt


def lines_of(ctx, fld, seeds, dt, steps, **kw):
    from paper_2606_02627_gb300 import api
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=steps, **kw)
    tr.upload_seeds(seeds)
    tr.trace()
    tr.check()
    out = tr.get_lines()
    torch.cuda.synchronize()
    return out


def same(a, b):
    assert torch.equal(a.offsets, b.offsets)
    assert torch.equal(a.vertices, b.vertices)
    assert torch.equal(a.status, b.status)


@pytest.mark.gpu
def test_tune_returns_a_candidate_and_caches_it(small, tmp_path):
    from paper_2606_02627_gb300 import api, autotune
    ctx, g, F, seeds, dt = small
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(3, 3, 3), dtype="f32", layout="cell8")
    fld.set_global(torch.from_numpy(F).cuda())
    cands = [(64, 4, 128, 0), (256, 3, 256, 0), (128, 6, 256, -1)]
    cache = str(tmp_path / "tune.json")
    log = []
    best = autotune.tune(ctx, fld, seeds, dt, 400, cands=cands, first=1500, cache=cache, log=log.append)
    assert best in [autotune.schedule_of(c) for c in cands]
    assert len(log) >= len(cands)
    log2 = []
    assert autotune.tune(ctx, fld, seeds, dt, 400, cands=cands, first=1500, cache=cache, log=log2.append) == best
    assert log2 == []                     # served from the cache
    # every schedule gives the same lines, bit for bit
    outs = [lines_of(ctx, fld, seeds, dt, 400, **sched)
            for sched in [best, {}] + [autotune.schedule_of(c) for c in cands]]
    for o in outs[1:]:
        same(o, outs[0])


@pytest.mark.gpu
def test_tune_structure_over_layouts_bricks_and_windows(small, tmp_path):
    from paper_2606_02627_gb300 import api, autotune
    ctx, g, F, seeds, dt = small
    src = torch.from_numpy(F).cuda()
    structs = [("cell8", (3, 3, 3), 0), ("tiled4", (2, 2, 2), 0), ("linear", (3, 3, 3), 0), ("cell8", (3, 3, 3), 4),
               ("cell8", (2, 2, 2), 1)]
    cands = [(256, 3, 256, 0), (128, 4, 128, -1)]
    cache = str(tmp_path / "structure.json")
    log = []
    choice = autotune.tune_structure(ctx, src, g, "f32", seeds, dt, 300, structs=structs, cands=cands, first=1000,
                                     cache=cache, log=log.append)
    assert (choice["layout"], tuple(choice["bricks"]), choice["brick_window"]) in structs
    assert choice["schedule"] in [autotune.schedule_of(c) for c in cands]
    assert any("structure" in l for l in log) and any("schedule" in l for l in log)
    log2 = []
    assert autotune.tune_structure(ctx, src, g, "f32", seeds, dt, 300, structs=structs, cands=cands, first=1000,
                                   cache=cache, log=log2.append) == choice
    assert log2 == []
    # every structure and schedule gives the same lines, bit for bit, and the
    # oracle's within the FP32 bound
    ref = None
    for lay, br, w in structs:
        fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=br, dtype="f32", layout=lay)
        fld.set_global(src)
        for c in cands:
            out = lines_of(ctx, fld, seeds, dt, 300, brick_window=w, **autotune.schedule_of(c))
            if ref is None:
                ref = out
            else:
                same(out, ref)
        fld.close()
    from tests.helpers import compare_lines
    sub = seeds[:500].cpu().numpy()
    want = oracle.trace_streamlines(F, g.origin, g.spacing, sub, dt, 300, eps=1e-6)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=tuple(choice["bricks"]), dtype="f32",
                    layout=choice["layout"])
    fld.set_global(src)
    got = lines_of(ctx, fld, seeds[:500].contiguous(), dt, 300, brick_window=choice["brick_window"],
                   **choice["schedule"])
    compare_lines(got, g, want, tol=1e-3)
