"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Inputs are seeded and synthetic; sizes keep the oracle to seconds while
spanning several bricks and ragged brick edges.  Tolerances (cells):
FP32 fields 1e-3 for every kernel (the stated bound after 1000 steps); the
compact storage types 2e-3 against the oracle on their own dequantised
samples (which isolates the arithmetic), and FX21 5e-2 against the oracle on
the FP32 field (the stated precision bound).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs
from tests.helpers import compare_lines, split_lines

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-3


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_02627_gb300 import api
    import __graft_entry__
    __graft_entry__.build()
    return api.Context(0)


def make_field(ctx, grid, F, bricks=(1, 1, 1), dtype="f32", layout="linear"):
    from paper_2606_02627_gb300 import api
    fld = api.Field(ctx, grid.dims, grid.origin, grid.spacing, bricks=bricks, dtype=dtype, layout=layout)
    fld.set_global(torch.from_numpy(np.ascontiguousarray(F)).cuda())
    return fld


def run(ctx, fld, seeds, dt, max_steps, kernel="persistent", **kw):
    from paper_2606_02627_gb300 import api
    tr = api.Tracer(ctx, fld, capacity=max(1, len(seeds)), dt=dt, max_steps=max_steps, kernel=kernel, **kw)
    tr.upload_seeds(torch.from_numpy(np.ascontiguousarray(seeds, dtype=np.float32)).cuda())
    tr.trace()
    tr.check()
    lines = tr.get_lines()
    torch.cuda.synchronize()
    return tr, lines


# ---------------------------------------------------------------- field store

@pytest.mark.parametrize("dtype,layout", [("f32", "linear"), ("bf16", "linear"), ("f16", "linear"),
                                          ("bf16", "tiled4"), ("f32", "tiled4"), ("f32", "cell8"),
                                          ("bf16", "cell8"), ("f16", "cell8"), ("fx21", "linear"),
                                          ("fx21", "cell8")])
def test_brick_store_matches_oracle_bit_exact(ctx, dtype, layout):
    g = inputs.cube_grid(19)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(4, n_modes=32, kmax=5)).numpy() * np.float32(7.0)
    F[3, 4, 5, 1] = np.nan
    F[0, 0, 0, 0] = np.float32(3e-9)
    bricks = (3, 2, 2)
    fld = make_field(ctx, g, F, bricks=bricks, dtype=dtype, layout=layout)
    code = {"f32": oracle.F32, "bf16": oracle.BF16, "f16": oracle.F16, "fx21": oracle.FX21}[dtype]
    scales, codes, _ = oracle.quantize_field(F, bricks, code, want_codes=True, want_dequant=False)
    n = oracle.brick_cells(g.dims, bricks)
    for bz in range(2):
        for by in range(2):
            for bx in range(3):
                b = (bz * 2 + by) * 3 + bx
                got, sc = fld.read_brick(bx, by, bz)
                if dtype == "f32":
                    ix = np.clip(bx * n[0] - 1 + np.arange(n[0] + 3), 0, 18)
                    iy = np.clip(by * n[1] - 1 + np.arange(n[1] + 3), 0, 18)
                    iz = np.clip(bz * n[2] - 1 + np.arange(n[2] + 3), 0, 18)
                    np.testing.assert_array_equal(got.view(np.uint32), F[np.ix_(iz, iy, ix)].view(np.uint32))
                elif dtype == "fx21":
                    assert sc == scales[b]
                    np.testing.assert_array_equal(got, codes[b])
                else:
                    assert sc == scales[b]
                    ref = codes[b]
                    nan_ref = (ref & 0x7FFF) > (0x7F80 if dtype == "bf16" else 0x7C00)
                    nan_got = (got & 0x7FFF) > (0x7F80 if dtype == "bf16" else 0x7C00)
                    np.testing.assert_array_equal(nan_got, nan_ref)
                    np.testing.assert_array_equal(got[~nan_ref], ref[~nan_ref])


def test_max_speed(ctx):
    g = inputs.cube_grid(33)
    F = inputs.abc_field(g)
    fld = make_field(ctx, g, F, bricks=(2, 2, 2))
    assert fld.max_speed() == pytest.approx(oracle.max_speed(F, g.spacing), rel=1e-6)
    glob = make_field(ctx, g, F, layout="global")
    assert glob.max_speed() == pytest.approx(oracle.max_speed(F, g.spacing), rel=1e-6)


# ---------------------------------------------------------------- analytic fields (plain method, one brick)

@pytest.mark.parametrize("kernel", ["persistent", "per_step", "per_seed"])
@pytest.mark.parametrize("which", ["rotation", "abc"])
def test_single_brick_analytic_fields(ctx, kernel, which):
    n = 64
    g = inputs.cube_grid(n)
    F = inputs.rotation_field(g) if which == "rotation" else inputs.abc_field(g)
    seeds = inputs.uniform_seeds(g, 1024, 0, lo_cells=1.0)
    dt = 0.25 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 500, eps=1e-6)
    fld = make_field(ctx, g, F, layout="global" if kernel == "per_seed" else "linear")
    _, lines = run(ctx, fld, seeds, dt, 500, kernel=kernel)
    st = compare_lines(lines, g, ref, tol=FP32_TOL)
    assert st["vertices"] > 100_000
    if kernel == "per_seed":
        # the plain kernel reads the global float3 array, the persistent one
        # its brick: the same samples and the same operations, so the same bits
        lin = make_field(ctx, g, F, layout="linear")
        _, pers = run(ctx, lin, seeds, dt, 500, kernel="persistent")
        assert torch.equal(lines.offsets, pers.offsets)
        assert torch.equal(lines.vertices, pers.vertices)
        assert torch.equal(lines.status, pers.status)


# ---------------------------------------------------------------- bricks invisible

@pytest.mark.parametrize("layout", ["linear", "tiled4", "cell8"])
def test_bricks_are_invisible_exhaustive_8cube(ctx, layout):
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(3)
    F = (0.4 * rng.standard_normal((9, 9, 9, 3))).astype(np.float32)
    ax = np.arange(0, 8.0001, 0.25)
    pts = np.stack(np.meshgrid(ax, ax[::4], ax[::2], indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    dt = 0.9 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, pts, dt, 40, eps=1e-6)
    fld = make_field(ctx, g, F, bricks=(2, 2, 2), layout=layout)
    _, lines = run(ctx, fld, pts, dt, 40)
    compare_lines(lines, g, ref, tol=1e-3, tie_cells=1e-4)
    # the decomposition is invisible to the arithmetic: one brick gives the same bits
    one = make_field(ctx, g, F, bricks=(1, 1, 1), layout=layout)
    _, lines1 = run(ctx, one, pts, dt, 40)
    assert torch.equal(lines.offsets, lines1.offsets)
    assert torch.equal(lines.vertices, lines1.vertices)
    assert torch.equal(lines.status, lines1.status)


@pytest.mark.parametrize("dtype,layout", [("f32", "linear"), ("bf16", "linear"), ("f16", "linear"),
                                          ("bf16", "cell8"), ("f32", "cell8"), ("fx21", "cell8")])
def test_bricked_equals_single_brick_bit_exact(ctx, dtype, layout):
    g = inputs.cube_grid(41)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(7, n_modes=64, kmax=2)).numpy()
    seeds = inputs.uniform_seeds(g, 3000, 7)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    out = []
    for bricks in [(1, 1, 1), (4, 4, 4), (3, 5, 2)]:
        fld = make_field(ctx, g, F, bricks=bricks, dtype=dtype, layout=layout)
        _, lines = run(ctx, fld, seeds, dt, 400, steps_per_round=13)
        out.append(lines)
    for o in out[1:]:
        assert torch.equal(o.offsets, out[0].offsets)
        if dtype in ("f16", "fx21"):
            # the tie bit depends on the exit margin, which moves with the decode
            assert torch.equal(o.status & 0x7F, out[0].status & 0x7F)
        else:
            assert torch.equal(o.status, out[0].status)
        if dtype in ("f16", "fx21"):
            # FP16 subnormal codes and FX21 codes round on a grid set by the brick
            # scale: a ghost copy may decode differently from its owner when the
            # two bricks' scales differ
            d = ((o.vertices - out[0].vertices).abs() / torch.tensor(g.spacing, device=o.vertices.device)).max()
            assert d.item() < (1e-3 if dtype == "f16" else 5e-2)
        else:
            assert torch.equal(o.vertices, out[0].vertices)


def test_fp32_layouts_and_kernels_give_the_same_bits(ctx):
    # FP32 samples are stored as given in every layout, and every kernel
    # interpolates them with the same operations in the same order: the
    # global float3 array (per-seed kernel), LINEAR and TILED4 bricks (lanes in
    # lockstep) and CELL8 records (decoupled lanes, and lockstep) give the same
    # lines bit for bit
    g = inputs.cube_grid(45)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(13, n_modes=64, kmax=3)).numpy()
    seeds = inputs.uniform_seeds(g, 3000, 13)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    runs = []
    for kernel, layout, bricks in (("per_seed", "global", (1, 1, 1)), ("persistent", "linear", (3, 2, 2)),
                                   ("persistent", "tiled4", (2, 2, 2)), ("persistent", "cell8", (3, 3, 1)),
                                   ("lockstep", "cell8", (1, 1, 1))):
        fld = make_field(ctx, g, F, bricks=bricks, layout=layout)
        _, lines = run(ctx, fld, seeds, dt, 500, kernel=kernel)
        runs.append(lines)
    for other in runs[1:]:
        assert torch.equal(other.offsets, runs[0].offsets)
        assert torch.equal(other.vertices, runs[0].vertices)
        assert torch.equal(other.status, runs[0].status)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "fx21"])
def test_decoupled_lanes_equal_lockstep_bit_exact(ctx, dtype):
    # CELL8 fields: the persistent kernel runs each lane's stages on its own
    # record copies; the lockstep kernel loads every sample with the whole
    # warp.  Same arithmetic, so the same bits, under any schedule.
    g = inputs.cube_grid(57)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(11, n_modes=64, kmax=3)).numpy()
    seeds = inputs.uniform_seeds(g, 4000, 11)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    for bricks, sched in [((4, 4, 4), dict(steps_per_round=13)), ((3, 5, 2), dict()),
                          ((1, 1, 1), dict(steps_per_round=7, drain_steps=3, block_size=64, blocks_per_sm=3))]:
        fld = make_field(ctx, g, F, bricks=bricks, dtype=dtype, layout="cell8")
        _, a = run(ctx, fld, seeds, dt, 600, kernel="persistent", **sched)
        _, b = run(ctx, fld, seeds, dt, 600, kernel="lockstep", **sched)
        assert torch.equal(a.offsets, b.offsets)
        assert torch.equal(a.vertices, b.vertices)
        assert torch.equal(a.status, b.status)
        assert torch.equal(a.margin, b.margin)


def test_uneven_bricks_match_undecomposed(ctx):
    g = inputs.Grid((23, 17, 30), (0.5, -1.0, 2.0), (0.25, 0.5, 0.125))
    F = inputs.turbulence_field(g, inputs.turbulence_modes(5, n_modes=48, kmax=4)).numpy()
    seeds = inputs.uniform_seeds(g, 600, 9)
    dt = 0.7 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 300, eps=1e-6)
    for bricks in [(3, 2, 5), (1, 4, 2), (5, 1, 1)]:
        fld = make_field(ctx, g, F, bricks=bricks)
        _, lines = run(ctx, fld, seeds, dt, 300, steps_per_round=7)
        compare_lines(lines, g, ref, tol=FP32_TOL)


# ---------------------------------------------------------------- turbulence, precision forms

@pytest.fixture(scope="module")
def turb64():
    # the shortest wavelength spans 32 cells, as on the 512^3 field with |k| <= 16
    g = inputs.cube_grid(129)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1, kmax=4)).numpy()
    seeds = inputs.uniform_seeds(g, 1500, 1)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 1000, eps=1e-6)
    return g, F, seeds, dt, ref


def test_rough_field_short_lines(ctx):
    # 4-cell wavelengths: strongly stretching flow, kept to 150 steps
    g = inputs.cube_grid(65)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(1)).numpy()
    seeds = inputs.uniform_seeds(g, 1500, 1)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 150, eps=1e-6)
    fld = make_field(ctx, g, F, bricks=(4, 4, 4))
    _, lines = run(ctx, fld, seeds, dt, 150)
    compare_lines(lines, g, ref, tol=FP32_TOL)


@pytest.mark.parametrize("layout", ["linear", "cell8"])
def test_turbulence_fp32_bricked_1000_steps(ctx, turb64, layout):
    g, F, seeds, dt, ref = turb64
    fld = make_field(ctx, g, F, bricks=(4, 4, 4), layout=layout)
    _, lines = run(ctx, fld, seeds, dt, 1000)
    st = compare_lines(lines, g, ref, tol=FP32_TOL)
    print("fp32", st["max_err"], st["p99"], st["ties"])


# The stated precision bound is 5e-2 cells against the FP64 oracle on the FP32
# field.  FX21 (21-bit fixed point in the same 8 bytes per sample) must meet it
# for every vertex of this field.  BF16 and FP16 are held to the arithmetic
# bound against the oracle on their own dequantised samples; their error
# against the FP32 field is reported here (this 1000-step, strongly stretching
# field amplifies their 8- and 11-bit mantissas beyond 5e-2) and asserted at
# the 99th percentile on the 1024^3 precision workload, where the stated bound
# holds (test_gpu_fullsize).
FX21_MAX_ERR = 5e-2


@pytest.mark.parametrize("dtype,layout", [("bf16", "linear"), ("f16", "linear"), ("bf16", "cell8"),
                                          ("f16", "cell8"), ("fx21", "linear"), ("fx21", "cell8")])
def test_turbulence_quantized(ctx, turb64, dtype, layout):
    g, F, seeds, dt, ref = turb64
    fld = make_field(ctx, g, F, bricks=(4, 4, 4), dtype=dtype, layout=layout)
    _, lines = run(ctx, fld, seeds, dt, 1000)
    code = {"bf16": oracle.BF16, "f16": oracle.F16, "fx21": oracle.FX21}[dtype]
    _, _, deq = oracle.quantize_field(F, (4, 4, 4), code)
    ref_q = oracle.trace_streamlines(deq, g.origin, g.spacing, seeds, dt, 1000, eps=1e-6)
    # the arithmetic: every line within 2e-3 cells of the oracle on the same stored (dequantised) samples
    st_q = compare_lines(lines, g, ref_q, tol=2e-3)
    # the precision form against the FP32-field oracle (common prefixes of every line)
    st = compare_lines(lines, g, ref, tol=1e9, tie_cells=0.5)
    print(dtype, layout, "vs dequantised", st_q["max_err"], "vs fp32 field max", st["max_err"], "p99", st["p99"])
    if dtype == "fx21":
        assert st["max_err"] <= FX21_MAX_ERR


# ---------------------------------------------------------------- step() and edge cases

@pytest.mark.parametrize("layout", ["linear", "cell8"])
def test_step_calls_equal_one_trace(ctx, turb64, layout):
    from paper_2606_02627_gb300 import api
    g, F, seeds, dt, ref = turb64
    fld = make_field(ctx, g, F, bricks=(3, 2, 2), layout=layout)
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=300)
    tr.upload_seeds(torch.from_numpy(seeds).cuda())
    steps = 0
    while True:
        active = tr.step(37)
        steps += 37
        if not active:
            break
        assert steps < 400
    lines = tr.get_lines()
    ref300 = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 300, eps=1e-6)
    compare_lines(lines, g, ref300, tol=FP32_TOL)


@pytest.mark.parametrize("layout,timed", [("linear", False), ("cell8", False), ("cell8", True)])
def test_round_cap_stops_with_consistent_partial_lines(ctx, turb64, layout, timed):
    # trace() stops when the rounds are all gone and nothing is left (Sec. 3.2);
    # a round cap below that stops it early with SG_ERR_ROUND_LIMIT.  The lines
    # written so far must read back consistently (every vertex the oracle's),
    # and calling trace() again continues them to the uncapped result.
    from paper_2606_02627_gb300 import _lib, api
    g, F, seeds, dt, _ = turb64
    ref300 = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 300, eps=1e-6)
    fld = make_field(ctx, g, F, bricks=(3, 2, 2), layout=layout)
    spr = 13
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=300, steps_per_round=spr, max_rounds=1)
    tr.upload_seeds(torch.from_numpy(seeds).cuda())

    def one_call():
        try:
            if timed:
                tr.trace_timed()
            else:
                tr.trace()
                tr.check()
            return True
        except _lib.StreamGBError as e:
            assert e.code == _lib.SG_ERR_ROUND_LIMIT, e
            return False

    assert not one_call()
    lines = tr.get_lines()
    torch.cuda.synchronize()
    st = lines.status.cpu().numpy() & 0x7F
    lens = lines.lengths().cpu().numpy()
    assert (st == 0).sum() > len(seeds) // 2                  # most lines are still running
    assert lens.max() <= spr + 1                               # one round: at most steps_per_round steps
    assert (lens[st == 0] >= 1).all()
    glines = split_lines(lines, g)
    for i in range(len(seeds)):
        r = ref300.line(i)
        k = min(len(glines[i]), len(r))
        if st[i] == 0:
            assert len(glines[i]) <= len(r)
        if k:
            assert np.abs(glines[i][:k] - r[:k]).max() <= FP32_TOL, i
    calls = 1
    while not one_call():
        calls += 1
        assert calls < 300
    final = tr.get_lines()
    compare_lines(final, g, ref300, tol=FP32_TOL)
    # the same bits as one uncapped trace with the same steps per round
    _, whole = run(ctx, fld, seeds, dt, 300, steps_per_round=spr)
    assert torch.equal(final.offsets, whole.offsets)
    assert torch.equal(final.vertices, whole.vertices)
    assert torch.equal(final.status, whole.status)


@pytest.mark.parametrize("layout,kernel,timed", [("cell8", "persistent", False), ("linear", "persistent", False),
                                                 ("cell8", "lockstep", False), ("cell8", "persistent", True)])
def test_brick_windows_give_the_same_bits(ctx, turb64, layout, kernel, timed):
    # the brick-major rounds policy advances the particles of a few bricks per
    # round and carries the others: the same arithmetic per particle, so the
    # same lines as advancing every brick each round
    from paper_2606_02627_gb300 import api
    g, F, seeds, dt, _ = turb64
    fld = make_field(ctx, g, F, bricks=(4, 4, 4), layout=layout)
    _, base = run(ctx, fld, seeds, dt, 400, kernel=kernel, steps_per_round=37)
    for w in (1, 5, 63):
        tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=400, kernel=kernel, steps_per_round=37,
                        brick_window=w)
        tr.upload_seeds(torch.from_numpy(seeds).cuda())
        if timed:
            ms, launches = tr.trace_timed()
        else:
            tr.trace()
            tr.check()
        lines = tr.get_lines()
        torch.cuda.synchronize()
        assert torch.equal(lines.offsets, base.offsets)
        assert torch.equal(lines.vertices, base.vertices)
        assert torch.equal(lines.status, base.status)


def test_oversized_blocks_are_refused_at_creation(ctx):
    # the kernels are built for at most 256 threads per CTA: a larger block is
    # an argument error when the tracer (or batch) is made, not a failed launch
    from paper_2606_02627_gb300 import _lib, api
    g = inputs.cube_grid(9)
    fld = make_field(ctx, g, inputs.uniform_field(g, (0.25, 0.0, 0.0)), layout="cell8")
    with pytest.raises(_lib.StreamGBError) as ei:
        api.Tracer(ctx, fld, capacity=16, dt=0.1, max_steps=10, block_size=512)
    assert ei.value.code == _lib.SG_ERR_INVALID_ARG
    with pytest.raises(_lib.StreamGBError) as ei:
        api.Batch(ctx, max_lines=64, slab_bytes=1 << 20, block_size=512)
    assert ei.value.code == _lib.SG_ERR_INVALID_ARG


def test_step_reports_active_lines(ctx):
    from paper_2606_02627_gb300 import api
    g = inputs.cube_grid(16)
    F = inputs.rotation_field(g)
    fld = make_field(ctx, g, F)
    tr = api.Tracer(ctx, fld, capacity=4, dt=0.01, max_steps=10)
    tr.upload_seeds(torch.tensor([[3.0, 3.0, 3.0], [2.0, 3.5, 1.0]]).cuda())
    assert tr.step(4) is True
    lines = tr.get_lines()
    assert lines.status.cpu().tolist() == [0, 0]
    assert lines.lengths().cpu().tolist() == [5, 5]
    assert tr.step(6) is False
    lines = tr.get_lines()
    assert lines.status.cpu().tolist() == [1, 1]
    assert lines.lengths().cpu().tolist() == [11, 11]


def test_edge_cases(ctx):
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    F = inputs.uniform_field(g, (0.25, 0.0, 0.0))
    F[2, 2, 6] = np.nan
    seeds = np.array([[1.0, 1.0, 1.0],        # runs to max steps
                      [8.0, 3.0, 3.0],        # on the upper face, flow outward: stops at once
                      [-0.5, 2.0, 2.0],       # outside: no vertex
                      [4.0, 2.0, 2.0],        # runs into the NaN sample
                      [0.0, 8.0, 8.0],        # corner
                      [4.0, 4.0, 4.0]], dtype=np.float32)
    ref = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, 1.0, 12, eps=1e-6)
    for kernel, layout, bricks in [("persistent", "linear", (2, 2, 2)), ("per_step", "linear", (2, 1, 3)),
                                   ("per_seed", "global", (1, 1, 1)), ("persistent", "cell8", (2, 2, 2)),
                                   ("lockstep", "cell8", (2, 1, 3))]:
        fld = make_field(ctx, g, F, bricks=bricks, layout=layout)
        for ms in (0, 1, 12):
            r = ref if ms == 12 else oracle.trace_streamlines(F, g.origin, g.spacing, seeds, 1.0, ms, eps=1e-6)
            _, lines = run(ctx, fld, seeds, 1.0, ms, kernel=kernel)
            compare_lines(lines, g, r, tol=1e-5)
            assert (lines.status.cpu().numpy() & 0x7F).tolist() == r.status.tolist()


def test_zero_field_and_empty_seeds(ctx):
    from paper_2606_02627_gb300 import api
    g = inputs.cube_grid(8)
    F = np.zeros((8, 8, 8, 3), np.float32)
    fld = make_field(ctx, g, F, bricks=(2, 2, 2), dtype="bf16")
    seeds = inputs.uniform_seeds(g, 50, 2)
    _, lines = run(ctx, fld, seeds, 0.1, 10)
    assert (lines.status.cpu().numpy() == 3).all()
    assert (lines.lengths().cpu().numpy() == 1).all()
    tr = api.Tracer(ctx, fld, capacity=10, dt=0.1, max_steps=10)
    tr.upload_seeds(torch.zeros((0, 3)).cuda())
    tr.trace()
    assert tr.sizes() == (0, 0)


def test_lines_to_pinned_host_and_total_steps(ctx, turb64):
    g, F, seeds, dt, ref = turb64
    from paper_2606_02627_gb300 import api
    fld = make_field(ctx, g, F, bricks=(4, 4, 4))
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=1000)
    tr.upload_seeds(torch.from_numpy(seeds))          # pageable host seeds
    tr.trace()
    host = tr.get_lines(device="pinned")
    torch.cuda.synchronize()
    dev = tr.get_lines()
    torch.cuda.synchronize()
    assert torch.equal(host.vertices, dev.vertices.cpu())
    assert torch.equal(host.offsets, dev.offsets.cpu())
    lens = dev.lengths().cpu().numpy()
    assert tr.total_steps() == int(np.maximum(lens - 1, 0).sum())
    compare_lines(dev, g, ref, tol=FP32_TOL)


def test_overlapped_readout_pipelined(ctx, turb64):
    """The host copy of trace k overlaps trace k+1 on the same tracer: every
    host result equals the synchronous device readout.  Four readouts in a
    row use the tracer's two staging buffers in turn; the fourth needs a
    larger second buffer than the second readout left."""
    g, F, seeds, dt, ref = turb64
    from paper_2606_02627_gb300 import api, _lib
    fld = make_field(ctx, g, F, bricks=(4, 4, 4), layout="cell8")
    tr = api.Tracer(ctx, fld, capacity=len(seeds), dt=dt, max_steps=1000)
    s = torch.cuda.current_stream()
    other = inputs.uniform_seeds(g, len(seeds) // 2, 7)
    dev_ref = []
    for sd in (seeds, other):
        tr.upload_seeds(sd)
        tr.trace()
        L = tr.get_lines()
        torch.cuda.synchronize()
        dev_ref.append((L.offsets.cpu(), L.vertices.cpu(), L.status.cpu(), L.margin.cpu()))
    outs = []
    pinned = [torch.from_numpy(sd).pin_memory() for sd in (seeds, other)]
    which = (0, 1, 0, 0)
    for k in which:
        tr.upload_seeds(pinned[k], stream=s)
        tr.trace(stream=s)
        outs.append(tr.get_lines_overlapped(stream=s))   # the next trace is enqueued before its copy is waited for
    tr.wait_lines(s)
    s.synchronize()
    for k, out in zip(which, outs):
        o, v, st, mg = dev_ref[k]
        assert torch.equal(out.offsets, o)
        assert torch.equal(out.vertices, v)
        assert torch.equal(out.status, st)
        assert torch.equal(out.margin, mg)
    compare_lines(outs[2], g, ref, tol=FP32_TOL)
    # reuse of the host buffers, and the empty trace
    tr.upload_seeds(torch.zeros((0, 3)).cuda())
    tr.trace()
    e = tr.get_lines_overlapped(out=outs[0])
    tr.wait_lines()
    torch.cuda.synchronize()
    assert e.offsets.tolist() == [0] and e.vertices.shape[0] == 0
    with pytest.raises(_lib.StreamGBError):             # pageable host memory is refused
        api.call("sg_tracer_get_lines_overlapped", tr.h, None, None, np.zeros(4, np.int64).ctypes.data,
                 None, None, None, None)


def test_invalid_arguments(ctx):
    from paper_2606_02627_gb300 import api, _lib
    g = inputs.cube_grid(8)
    with pytest.raises(_lib.StreamGBError):
        api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(8, 1, 1))
    fld = make_field(ctx, g, np.zeros((8, 8, 8, 3), np.float32))
    with pytest.raises(_lib.StreamGBError):
        api.Tracer(ctx, fld, capacity=4, dt=0.0, max_steps=10)
    with pytest.raises(_lib.StreamGBError):
        api.Tracer(ctx, fld, capacity=4, dt=0.1, max_steps=10, kernel="per_seed")
    tr = api.Tracer(ctx, fld, capacity=4, dt=0.1, max_steps=10)
    with pytest.raises(_lib.StreamGBError):
        tr.upload_seeds(torch.zeros((5, 3)).cuda())


# ---------------------------------------------------------------- streaklines

def test_streaklines_match_oracle(ctx):
    from paper_2606_02627_gb300 import api
    n = 33
    g = inputs.cube_grid(n)
    modes = inputs.turbulence_modes(3, n_modes=64, kmax=6)
    n_slices = 12
    slices = np.stack([inputs.turbulence_field(g, modes, time_slice=s, n_slices=n_slices).numpy()
                       for s in range(n_slices)])
    vref = max(oracle.max_speed(slices[s], g.spacing) for s in range(n_slices))
    dt = 0.5 / vref
    sdt = dt                           # one advection step per slice interval
    R, inj, steps = 40, 8, n_slices - 1
    release = inputs.uniform_seeds(g, R, 4, lo_cells=2.0)
    ref = oracle.trace_streaklines(slices, g.origin, g.spacing, sdt, release, dt, steps, inj)
    fld = api.Field(ctx, g.dims, g.origin, g.spacing, bricks=(2, 2, 2), n_slots=3, slice_dt=sdt)
    pinned = [torch.from_numpy(slices[s]).pin_memory() for s in range(n_slices)]
    side = torch.cuda.Stream()
    tr = api.Tracer(ctx, fld, capacity=R, dt=dt, mode="streakline", inject_steps=inj)
    with torch.cuda.stream(side):
        fld.stream_slice(0, pinned[0], stream=side)
        fld.stream_slice(1, pinned[1], stream=side)
    tr.upload_seeds(torch.from_numpy(release).cuda())
    for j in range(1, steps + 1):
        if j + 1 < n_slices:
            # the library orders the overwrite of a slot after the last step that read it
            fld.stream_slice(j + 1, pinned[j + 1], stream=side)
        tr.step(1, sync=False)
    lines = tr.get_lines()
    torch.cuda.synchronize()
    # expected lines from the oracle's particles: runs of live particles in birth order
    idx = split_lines(lines, g)
    src = lines.source.cpu().numpy()
    k = 0
    for r in range(R):
        live = ref.status[r] == oracle.ACTIVE
        b = 0
        while b < inj:
            if not live[b]:
                b += 1
                continue
            e = b
            while e < inj and live[e]:
                e += 1
            assert src[k] == r
            np.testing.assert_allclose(idx[k], ref.pos[r, b:e], atol=1e-4)
            k += 1
            b = e
    assert k == len(idx)
