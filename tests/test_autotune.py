"""Schedule autotuner (successive halving over the persistent kernel's
schedule): candidate grid on the CPU; on the GPU, the tuner returns one of the
candidates, caches it per problem shape, and a schedule changes no bit of the
lines (the schedule decides only which lane advances which particle when).
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


@pytest.mark.gpu
def test_tune_returns_a_candidate_and_caches_it(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api, autotune
    ctx = api.Context(0)
    g = inputs.cube_grid(49)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(21, n_modes=48, kmax=3)).numpy()
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(3, 3, 3), dtype="f32", layout="cell8")
    fld.set_global(torch.from_numpy(F).cuda())
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 6000, 21)).cuda()
    dt = 0.5 / oracle.max_speed(F, g.spacing)
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
    outs = []
    for sched in [best, {}] + [autotune.schedule_of(c) for c in cands]:
        tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=400, **sched)
        tr.upload_seeds(seeds)
        tr.trace()
        tr.check()
        outs.append(tr.get_lines())
    for o in outs[1:]:
        assert torch.equal(o.offsets, outs[0].offsets)
        assert torch.equal(o.vertices, outs[0].vertices)
        assert torch.equal(o.status, outs[0].status)
