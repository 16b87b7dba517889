"""Unstructured fields on the GPU (hexahedra, tetrahedra, prisms, pyramids)
against the FP64 oracle: point location and interpolation at random points,
and streamlines through jittered meshes of a smooth turbulence field (every
vertex within 1e-3 cells, statuses and lengths equal up to boundary ties)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs
from tests.helpers import compare_lines

pytestmark = pytest.mark.gpu

KINDS = ["hex", "tet", "prism", "pyramid"]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import api
    return api.Context(0)


@pytest.fixture(scope="module")
def turb():
    # the modes' shortest wavelength spans the grid: a smooth flow, in which a
    # 1e-6 change of a seed moves no vertex by more than ~1e-4 cells in 300 steps
    h = 2 * np.pi / 20
    g = inputs.Grid((21, 19, 17), (0.0, 0.0, 0.0), (h, h, h))
    F = inputs.turbulence_field(g, inputs.turbulence_modes(71, n_modes=48, kmax=1)).numpy()
    return g, F


@pytest.mark.parametrize("kind", KINDS)
def test_umesh_sample_matches_oracle(ctx, kind):
    from paper_2606_02627_gb300 import api
    g = inputs.Grid((9, 8, 7), (1.0, -2.0, 0.5), (0.5, 0.75, 1.0))
    F = inputs.turbulence_field(g, inputs.turbulence_modes(72, n_modes=16, kmax=2)).numpy()
    m = inputs.grid_mesh(g, F, kind=kind, jitter=0.2, seed=9)
    mesh = api.UMesh(ctx, m)
    lo = np.asarray(g.origin) - 0.2
    hi = np.asarray(g.origin) + np.asarray(g.spacing) * (np.asarray(g.dims) - 1) + 0.2
    pts = (lo + (hi - lo) * inputs.uniform(9, 2, 6000).reshape(-1, 3)).astype(np.float32)
    v_ref, c_ref = oracle.umesh_sample(m, pts.astype(np.float64), tau=1e-5)
    v, c = mesh.sample(torch.from_numpy(pts))
    v, c = v.cpu().numpy(), c.cpu().numpy()
    inside = c_ref >= 0
    # points within 1e-4 of the mesh boundary may fall either way
    box_lo = np.asarray(g.origin) + 1e-4
    box_hi = np.asarray(g.origin) + np.asarray(g.spacing) * (np.asarray(g.dims) - 1) - 1e-4
    clear = ((pts > box_lo) & (pts < box_hi)).all(1) | ~((pts >= box_lo - 2e-4) & (pts <= box_hi + 2e-4)).all(1)
    assert ((c >= 0) == inside)[clear].all()
    both = inside & (c >= 0)
    scale = np.abs(v_ref[both]).max()
    np.testing.assert_allclose(v[both], v_ref[both], atol=2e-5 * scale)
    assert np.isnan(v[c < 0]).all()


@pytest.mark.parametrize("kind", KINDS)
def test_umesh_trace_matches_oracle(ctx, turb, kind):
    from paper_2606_02627_gb300 import api
    g, F = turb
    m = inputs.grid_mesh(g, F, kind=kind, jitter=0.15, seed=11)
    mesh = api.UMesh(ctx, m)
    seeds = inputs.uniform_seeds(g, 300, 11)
    seeds[:3] = np.float32(-3.0)                        # OUT
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_umesh(m, seeds.astype(np.float64), dt, 300, tau=1e-5)
    lines = mesh.trace(torch.from_numpy(seeds), dt, 300)
    st = compare_lines(lines, g, ref_index_space(ref, g), tol=1e-3)
    print(kind, st["max_err"], st["p99"], st["ties"])
    assert st["vertices"] > 300 * 20


def ref_index_space(ref, g):
    """Oracle world-space Lines as index-space Lines (what compare_lines reads)."""
    org, sp = np.asarray(g.origin), np.asarray(g.spacing)

    class R:
        pass
    r = R()
    r.length, r.status, r.margin = ref.length, ref.status, ref.margin
    r.line = lambda i: (ref.line(i) - org) / sp
    return r


def test_umesh_edge_cases(ctx):
    from paper_2606_02627_gb300 import api
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    m = inputs.grid_mesh(g, inputs.uniform_field(g, (0.25, 0.0, 0.0)), kind="tet", jitter=0.2, seed=2)
    mesh = api.UMesh(ctx, m)
    seeds = np.array([[1.0, 4.3, 3.7], [-1.0, 2.0, 2.0], [8.0, 3.0, 3.0]], dtype=np.float32)
    for ms in (0, 1, 100):
        ref = oracle.trace_umesh(m, seeds.astype(np.float64), 1.0, ms, tau=1e-5)
        lines = mesh.trace(torch.from_numpy(seeds), 1.0, ms)
        assert lines.lengths().cpu().tolist() == ref.length.tolist()
        assert (lines.status.cpu().numpy() & 0x7F).tolist() == ref.status.tolist()
    assert lines.vertices.shape[0] == 29 + 0 + 1
    np.testing.assert_allclose(lines.vertices[:29, 0].cpu().numpy(), 1.0 + 0.25 * np.arange(29), atol=1e-5)
    with pytest.raises(api.L.StreamGBError):
        bad = dict(m)
        bad["cell_types"] = m["cell_types"].copy()
        bad["cell_types"][0] = 7
        api.UMesh(ctx, bad)


def test_umesh_trace_on_a_side_stream_equals_default_stream(ctx, turb):
    # the trace, its compaction and its buffers all live on the stream the
    # caller passes; two traces on two streams at once must not mix
    from paper_2606_02627_gb300 import api
    g, F = turb
    m = inputs.grid_mesh(g, F, kind="hex", jitter=0.15, seed=12)
    mesh = api.UMesh(ctx, m)
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 500, 12))
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    ref = mesh.trace(seeds, dt, 200)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = mesh.trace(seeds, dt, 200, stream=s1)
    b = mesh.trace(seeds[:250], dt, 150, stream=s2)
    s1.synchronize()
    s2.synchronize()
    for got in (a,):
        assert torch.equal(got.offsets, ref.offsets)
        assert torch.equal(got.vertices, ref.vertices)
        assert torch.equal(got.status, ref.status)
    alone = mesh.trace(seeds[:250], dt, 150)
    torch.cuda.synchronize()
    assert torch.equal(b.offsets, alone.offsets)
    assert torch.equal(b.vertices, alone.vertices)


def test_umesh_round_caps_cut_lines_at_their_prefix(ctx):
    """The trace runs in rounds of at most 128 steps per particle.  Capped at
    m steps, around and across those round boundaries, every line is the
    first m + 1 vertices of the uncapped line, bit for bit, with its status
    where it stopped earlier and MAXSTEPS otherwise.  Solid-body rotation
    keeps the lines in the domain, so they run to the cap."""
    from paper_2606_02627_gb300 import api
    g = inputs.cube_grid(25)
    F = inputs.rotation_field(g)
    m = inputs.grid_mesh(g, F, kind="hex", jitter=0.1, seed=3)
    mesh = api.UMesh(ctx, m)
    seeds = torch.from_numpy(inputs.uniform_seeds(g, 256, 5, lo_cells=7.0, hi_cells=17.0))
    dt = 0.25 / oracle.max_speed(F, g.spacing)
    full = mesh.trace(seeds, dt, 600)
    torch.cuda.synchronize()
    f_off, f_v = full.offsets.cpu().numpy(), full.vertices.cpu().numpy()
    f_len, f_st = np.diff(f_off), full.status.cpu().numpy() & 0x7F
    assert (f_len == 601).sum() > 200                            # most lines run to the cap
    for ms in (127, 128, 129, 255, 256, 257):
        cap = mesh.trace(seeds, dt, ms)
        torch.cuda.synchronize()
        c_off, c_v = cap.offsets.cpu().numpy(), cap.vertices.cpu().numpy()
        c_len, c_st = np.diff(c_off), cap.status.cpu().numpy() & 0x7F
        np.testing.assert_array_equal(c_len, np.minimum(f_len, ms + 1))
        for i in range(len(c_len)):
            assert np.array_equal(c_v[c_off[i]:c_off[i + 1]], f_v[f_off[i]:f_off[i] + c_len[i]]), (ms, i)
        stopped = f_len <= ms                                      # ended before the cap in both
        assert (c_st[stopped] == f_st[stopped]).all()
        assert (c_st[~stopped] == 1).all()                          # SG_LINE_MAXSTEPS
