"""Partition over data on the GPU: ranks emulated as tracers in one process.

Each rank's tracer owns a share of the bricks (pod.partition_bricks), advects
only its own particles and hands the others to their owners between rounds
(sg_tracer_pod_*); pod.LocalTransport moves the records between the tracers
(device copies, no kernel of one rank waits on another's).  The merged lines
must equal an undivided trace bit for bit: the per-particle arithmetic is the
same whichever rank runs it.  The exchange between processes (all-to-all-v,
reductions) is tested on CPU ranks in test_pod_cpu.py.
"""
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


@pytest.mark.parametrize("layout,kernel,world", [("cell8", "persistent", 1), ("cell8", "persistent", 2),
                                                 ("cell8", "persistent", 4), ("linear", "persistent", 3),
                                                 ("cell8", "lockstep", 2)])
def test_pod_equals_undivided_trace(ctx, layout, kernel, world):
    from paper_2606_02627_gb300 import api, pod
    g = inputs.cube_grid(65)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(61, n_modes=64, kmax=2)).numpy()
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 3000, 61)).cuda()
    seeds[:5] = -4.0
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    bricks = (4, 4, 4)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=bricks, layout=layout)
    fld.set_global(torch.from_numpy(F).cuda())
    ref_tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=500, kernel=kernel, steps_per_round=40)
    ref_tr.upload_seeds(seeds)
    ref_tr.trace()
    ref = ref_tr.get_lines()
    owner = pod.partition_bricks(bricks, world)
    engines = []
    for r in range(world):
        tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=500, kernel=kernel, steps_per_round=40)
        engines.append(pod.GpuEngine(tr, owner, r, world))
        tr.upload_seeds(seeds)
    rounds = pod.LocalTransport.trace_local(engines)
    assert rounds >= (1 if world == 1 else 3)
    for e in engines:
        got = e.tr.get_lines()
        assert torch.equal(got.offsets, ref.offsets)
        assert torch.equal(got.vertices, ref.vertices)
        assert torch.equal(got.status, ref.status)
        assert torch.equal(got.margin, ref.margin)
        assert e.tr.total_steps() == ref_tr.total_steps()
    # a partitioned tracer refuses the undivided calls
    with pytest.raises(api.L.StreamGBError):
        engines[0].tr.trace()
