"""Backward and bidirectional streamlines, and the seed-shape kernels, on the GPU.

* A backward tracer matches the FP64 oracle run with -dt (FP32 tolerance).
* A bidirectional tracer's line i equals a forward tracer's line i and its
  line n + i a backward tracer's line i, bit for bit (each lane takes its
  line's direction; the arithmetic is the same), for the persistent
  (decoupled and lockstep), Listing-1 and per-seed kernels.
* The joined polylines are the backward line reversed (seed once) followed by
  the forward line, element for element, with the seed's index; OUT seeds
  give empty polylines; against the oracle's two directions composed the
  same way, within the FP32 tolerance.
* The seed-shape kernels reproduce their stated formulas bit for bit
  (double arithmetic rounded once to float32; SplitMix64 for the box).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs
from tests.helpers import compare_lines

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-3


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    return api.Context(0)


@pytest.fixture(scope="module")
def turb():
    g = inputs.cube_grid(65)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(41, n_modes=64, kmax=2)).numpy()
    seeds = inputs.uniform_seeds(g, 1500, 41)
    seeds[:7] = np.float32(-1.0)                 # OUT seeds
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    return g, F, seeds, dt


def make_field(ctx, g, F, bricks, layout):
    from paper_2606_02627_gb300 import api
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=bricks, dtype="f32", layout=layout)
    fld.set_global(torch.from_numpy(np.ascontiguousarray(F)).cuda())
    return fld


def trace(ctx, fld, seeds, dt, ms, direction, kernel="persistent"):
    from paper_2606_02627_gb300 import api
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=ms, kernel=kernel, direction=direction,
                    steps_per_round=37)
    tr.upload_seeds(torch.from_numpy(seeds).cuda())
    tr.trace()
    tr.check()
    return tr


def test_backward_matches_oracle(ctx, turb):
    g, F, seeds, dt = turb
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, -dt, 800, eps=1e-6)
    for layout, kernel in (("cell8", "persistent"), ("linear", "persistent")):
        fld = make_field(ctx, g, F, (3, 2, 4), layout)
        lines = trace(ctx, fld, seeds, dt, 800, "backward", kernel).get_lines()
        compare_lines(lines, g, ref, tol=FP32_TOL)


def _slice(lines, a, b):
    off = lines.offsets.cpu()
    o = off[a:b + 1]
    return (o - o[0]), lines.vertices.cpu()[int(o[0]):int(o[-1])], lines.status.cpu()[a:b], lines.margin.cpu()[a:b]


@pytest.mark.parametrize("layout,kernel", [("cell8", "persistent"), ("cell8", "lockstep"), ("linear", "per_step"),
                                           ("global", "per_seed")])
def test_both_directions_equal_one_direction_tracers(ctx, turb, layout, kernel):
    g, F, seeds, dt = turb
    n = len(seeds)
    fld = make_field(ctx, g, F, (1, 1, 1) if layout == "global" else (2, 3, 2), layout)
    both = trace(ctx, fld, seeds, dt, 300, "both", kernel).get_lines()
    assert len(both.status) == 2 * n
    for k, d in ((0, "forward"), (1, "backward")):
        one = trace(ctx, fld, seeds, dt, 300, d, kernel).get_lines()
        o, v, s, m = _slice(both, k * n, (k + 1) * n)
        assert torch.equal(o, one.offsets.cpu())
        assert torch.equal(v, one.vertices.cpu())
        assert torch.equal(s, one.status.cpu())
        assert torch.equal(m, one.margin.cpu())
    src = both.source.cpu().numpy()
    assert (src == np.concatenate([np.arange(n), np.arange(n)])).all()


def test_joined_lines(ctx, turb):
    g, F, seeds, dt = turb
    n = len(seeds)
    fld = make_field(ctx, g, F, (2, 2, 2), "cell8")
    tr = trace(ctx, fld, seeds, dt, 400, "both")
    lines = tr.get_lines()
    J = tr.get_joined()
    off = lines.offsets.cpu().numpy()
    vert = lines.vertices.cpu().numpy()
    joff = J.offsets.cpu().numpy()
    jv = J.vertices.cpu().numpy()
    sv = J.seed_vertex.cpu().numpy()
    assert len(joff) == n + 1 and joff[0] == 0
    for i in range(n):
        f = vert[off[i]:off[i + 1]]
        b = vert[off[n + i]:off[n + i + 1]]
        got = jv[joff[i]:joff[i + 1]]
        if len(f) == 0:
            assert len(b) == 0 and len(got) == 0 and sv[i] == -1
            continue
        want = np.concatenate([b[1:][::-1], f])
        assert np.array_equal(got, want)
        assert sv[i] == len(b) - 1
        assert np.array_equal(got[sv[i]], seeds[i])
    assert tr.total_steps() == int(np.maximum(np.diff(off) - 1, 0).sum())
    # against the oracle's two directions composed the same way
    rf = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 400, eps=1e-6)
    rb = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, -dt, 400, eps=1e-6)
    compare_lines(lines, g, _concat(rf, rb), tol=FP32_TOL)


class _Both:
    """Oracle Lines of both directions stacked as lines 0..n-1, n..2n-1."""

    def __init__(self, a, b):
        self.a, self.b, self.n = a, b, len(a.length)
        self.length = np.concatenate([a.length, b.length])
        self.status = np.concatenate([a.status, b.status])
        self.margin = np.concatenate([a.margin, b.margin])

    def line(self, i):
        return self.a.line(i) if i < self.n else self.b.line(i - self.n)


def _concat(a, b):
    return _Both(a, b)


def test_joined_edge_cases(ctx):
    from paper_2606_02627_gb300 import api
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    F = inputs.uniform_field(g, (0.25, 0.0, 0.0))
    seeds = np.array([[4.0, 4.0, 4.0], [-1.0, 2.0, 2.0], [0.0, 3.0, 3.0], [8.0, 3.0, 3.0]], dtype=np.float32)
    fld = make_field(ctx, g, F, (2, 2, 2), "cell8")
    for ms in (0, 1, 40):
        tr = trace(ctx, fld, seeds, 1.0, ms, "both")
        J = tr.get_joined()
        lens = J.lengths().cpu().tolist()
        sv = J.seed_vertex.cpu().tolist()
        rf = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, 1.0, ms, eps=1e-6)
        rb = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, -1.0, ms, eps=1e-6)
        for i in range(len(seeds)):
            if rf.length[i] == 0:
                assert lens[i] == 0 and sv[i] == -1
            else:
                assert lens[i] == rf.length[i] + rb.length[i] - 1
                assert sv[i] == rb.length[i] - 1
    # joined readback needs a bidirectional tracer; streaklines are forward only
    one = trace(ctx, fld, seeds, 1.0, 5, "forward")
    with pytest.raises(api.L.StreamGBError):
        one.get_joined()


def test_seed_shape_kernels(ctx):
    from paper_2606_02627_gb300 import api
    a, b = np.array([0.5, -2.0, 3.25]), np.array([7.0, 1.5, -0.125])
    for n in (1, 2, 17, 100_003):
        got = api.seeds_rake(a, b, n).cpu().numpy()
        t = np.arange(n, dtype=np.float64) / (n - 1) if n > 1 else np.zeros(1)
        want = (a[None, :] + (b - a)[None, :] * t[:, None]).astype(np.float32)
        assert np.array_equal(got, want)
    o, u, v = np.array([1.0, 2.0, 3.0]), np.array([0.5, 0.0, 0.25]), np.array([0.0, -1.5, 0.75])
    for nu, nv in ((1, 1), (3, 1), (1, 4), (37, 29)):
        got = api.seeds_plane(o, u, v, nu, nv).cpu().numpy()
        s = np.arange(nu, dtype=np.float64) / (nu - 1) if nu > 1 else np.zeros(1)
        tt = np.arange(nv, dtype=np.float64) / (nv - 1) if nv > 1 else np.zeros(1)
        S, T = np.meshgrid(s, tt, indexing="xy")
        want = ((o[None, :] + u[None, :] * S.reshape(-1, 1)) + v[None, :] * T.reshape(-1, 1)).astype(np.float32)
        assert np.array_equal(got, want)
    lo, hi = np.array([-3.0, 0.25, 10.0]), np.array([5.0, 0.75, 12.5])
    for n, seed, stream in ((1, 0, 0), (1000, 7, 3), (250_000, 123456789, 1)):
        got = api.seeds_box(lo, hi, n, seed, stream).cpu().numpy()
        u01 = inputs.uniform(seed, stream, 3 * n).reshape(n, 3)
        want = (lo[None, :] + (hi - lo)[None, :] * u01).astype(np.float32)
        assert np.array_equal(got, want)
        assert (got >= lo.astype(np.float32)).all() and (got <= hi.astype(np.float32)).all()
    assert api.seeds_rake(a, b, 0).shape == (0, 3)
    with pytest.raises(api.L.StreamGBError):
        api.seeds_rake(a, b, -1)
