"""Pins of the FP64 oracle against closed forms, brute force and library routines.

Each test checks the oracle against something other than itself, so that a
dropped term, a wrong sign or index, or a transposed operand in oracle.c
fails at least one of them:

* uniform flow: exact straight lines and the exact exit step (dyadic values);
* solid-body rotation: the discrete RK4 closed form R(i theta)^n (trilinear
  interpolation is exact for linear fields);
* affine fields: the RK4 polynomial of the homogeneous matrix, and
  convergence to the matrix exponential at fourth order;
* ABC flow (analytic sampler): observed order 4 +- 0.3;
* trilinear interpolation: brute-force sum of hat functions over a 4^3 grid;
* quantisation: bit patterns from torch (bf16) and numpy (fp16) conversions;
* termination rules, brick ownership and streakline time interpolation.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2606_02627_gb300 import inputs


def unit_grid(n):
    """index space == world space (origin 0, spacing 1)."""
    return inputs.Grid((n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


# ---------------------------------------------------------------- uniform flow

def test_uniform_flow_exact_line_and_exit():
    g = unit_grid(17)
    F = inputs.uniform_field(g, (1.0, 0.0, 0.0))
    seed = np.array([[2.0, 5.5, 7.25]])
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seed, dt=0.25, max_steps=500)
    # p_n = 2 + n/4; the step from x = 16 has its first stage point at 16.125 > 16
    assert L.status[0] == oracle.EXIT
    assert L.length[0] == 57
    xs = 2.0 + 0.25 * np.arange(57)
    np.testing.assert_array_equal(L.line(0)[:, 0], xs)
    np.testing.assert_array_equal(L.line(0)[:, 1], 5.5)
    np.testing.assert_array_equal(L.line(0)[:, 2], 7.25)
    assert L.margin[0] == 0.125


def _exact_exit_steps(p0, k, hi):
    """Number of steps before a stage point p + c k (c in 1/2, 1) leaves [0, hi]."""
    p = [Fraction(x) for x in p0]
    k = [Fraction(x) for x in k]
    n = 0
    while True:
        for c in (Fraction(1, 2), Fraction(1)):
            q = [p[a] + c * k[a] for a in range(3)]
            if any(x < 0 or x > hi[a] for a, x in enumerate(q)):
                return n
        p = [p[a] + k[a] for a in range(3)]
        n += 1


@pytest.mark.parametrize("u,spacing,seed", [
    ((0.5, -0.25, 0.125), (0.5, 0.25, 1.0), (3.0, 20.0, 1.5)),
    ((-1.0, 0.0, 0.0), (1.0, 1.0, 1.0), (9.0, 0.0, 0.0)),
    ((0.0, 0.0, 2.0), (1.0, 1.0, 0.5), (4.0, 4.0, 0.0)),
])
def test_uniform_flow_anisotropic_spacing(u, spacing, seed):
    n = 33
    g = inputs.Grid((n, n, n), (0.0, 0.0, 0.0), spacing)
    F = inputs.uniform_field(g, u)
    dt = 0.125
    seed_w = np.array([[g.origin[a] + spacing[a] * seed[a] for a in range(3)]])
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seed_w, dt=dt, max_steps=10_000)
    k = [dt * u[a] / spacing[a] for a in range(3)]   # cells per step
    steps = _exact_exit_steps(seed, k, [n - 1] * 3)
    assert L.status[0] == oracle.EXIT
    assert L.length[0] == steps + 1
    expect = np.array(seed)[None, :] + np.arange(steps + 1)[:, None] * np.array(k)[None, :]
    np.testing.assert_array_equal(L.line(0), expect)


# ---------------------------------------------------------------- rotation

def _rk4_poly(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def test_rotation_discrete_closed_form():
    n = 64
    g = unit_grid(n)
    c = (n - 1) / 2.0                       # 31.5: samples are exact half-integers
    F = inputs.rotation_field(g, center=(c, c, c))
    theta = 0.05
    seeds = np.array([[40.0, c, 10.0], [c, 12.25, 50.0], [20.5, 44.0, 0.0]])
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt=theta, max_steps=300)
    R = _rk4_poly(1j * theta)
    # |R(i theta)|^2 = 1 - theta^6/72 + theta^8/576
    assert abs(abs(R) ** 2 - (1 - theta ** 6 / 72 + theta ** 8 / 576)) < 1e-15
    for i in range(3):
        assert L.status[i] == oracle.MAXSTEPS and L.length[i] == 301
        z0 = (seeds[i, 0] - c) + 1j * (seeds[i, 1] - c)
        zn = z0 * R ** np.arange(301)
        line = L.line(i)
        np.testing.assert_allclose(line[:, 0] - c, zn.real, atol=1e-10)
        np.testing.assert_allclose(line[:, 1] - c, zn.imag, atol=1e-10)
        np.testing.assert_array_equal(line[:, 2], seeds[i, 2])
        # the radius shrinks by |R| per step, and differs from the circle by O(theta^6)
        r = np.hypot(line[:, 0] - c, line[:, 1] - c)
        np.testing.assert_allclose(r, abs(z0) * abs(R) ** np.arange(301), rtol=1e-12)


# ---------------------------------------------------------------- affine fields

A_LIN = np.array([[-1 / 16, -1 / 2, 0.0], [1 / 2, -1 / 16, 1 / 32], [0.0, -1 / 32, -1 / 8]])


def _affine_setup(n=64):
    g = unit_grid(n)
    c = np.array([31.5, 31.5, 31.5])
    b = -A_LIN @ c
    F = inputs.linear_field(g, A_LIN, b)
    # exactly representable: A has entries k/32, grid points are integers
    np.testing.assert_array_equal(F.astype(np.float64), inputs.linear_field(g, A_LIN, b, dtype=np.float64))
    Ah = np.zeros((4, 4))
    Ah[:3, :3] = A_LIN
    Ah[:3, 3] = b
    return g, F, Ah


def test_affine_field_rk4_polynomial():
    g, F, Ah = _affine_setup()
    dt = 0.1
    seeds = np.array([[40.0, 30.0, 45.0], [25.0, 36.0, 20.0]])
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt=dt, max_steps=200)
    Z = dt * Ah
    P = np.eye(4) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    for i in range(2):
        assert L.status[i] == oracle.MAXSTEPS
        ph = np.append(seeds[i], 1.0)
        for step in range(201):
            np.testing.assert_allclose(L.line(i)[step], ph[:3], atol=1e-9)
            ph = P @ ph


def test_affine_field_converges_to_matrix_exponential_at_order_4():
    from scipy.linalg import expm
    g, F, Ah = _affine_setup()
    seed = np.array([[40.0, 30.0, 45.0]])
    T = 4.0
    errs = []
    for dt in (0.4, 0.2, 0.1):
        nsteps = int(round(T / dt))
        L = oracle.trace_streamlines(F, g.origin, g.spacing, seed, dt=dt, max_steps=nsteps)
        exact = (expm(T * Ah) @ np.append(seed[0], 1.0))[:3]
        errs.append(np.abs(L.line(0)[-1] - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 < o < 4.3 for o in orders), orders


# ---------------------------------------------------------------- ABC order

def test_abc_rk4_order_four():
    dims = (1 << 20,) * 3
    h = 2 * math.pi / 63
    origin = (-h * (1 << 19),) * 3
    seeds = np.array([[1.0, 2.0, 3.0], [4.0, 0.5, 5.5]])
    T = 2.0

    def run(dt):
        nsteps = int(round(T / dt))
        L = oracle.trace_abc(dims, origin, (h, h, h), seeds, dt, nsteps)
        assert (L.status == oracle.MAXSTEPS).all()
        return np.array([L.line(i)[-1] for i in range(len(seeds))]) * h

    ref = run(0.1 / 64)
    errs = [np.abs(run(dt) - ref).max() for dt in (0.1, 0.05, 0.025)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 < o < 4.3 for o in orders), orders


# ---------------------------------------------------------------- trilinear brute force

def _hat_sum(F, p):
    nz, ny, nx, _ = F.shape
    v = np.zeros(3)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                w = max(0.0, 1 - abs(p[0] - i)) * max(0.0, 1 - abs(p[1] - j)) * max(0.0, 1 - abs(p[2] - k))
                v += w * F[k, j, i].astype(np.float64)
    return v


def test_trilinear_equals_hat_function_sum_on_4cube():
    rng = np.random.default_rng(5)
    F = rng.standard_normal((4, 4, 4, 3)).astype(np.float32)
    pts = list(rng.uniform(0, 3, size=(40, 3)))
    special = [0.0, 0.5, 1.0, 2.0, 2.75, 3.0]
    pts += [np.array([a, b, c]) for a in special for b in special[::2] for c in (0.0, 3.0, 1.5)]
    pts = np.array(pts)
    got = oracle.sample(F, pts)
    for p, v in zip(pts, got):
        np.testing.assert_allclose(v, _hat_sum(F, p), rtol=0, atol=1e-13)


def test_trajectories_on_random_4cube_match_longdouble_bruteforce():
    rng = np.random.default_rng(11)
    F = (0.3 * rng.standard_normal((4, 4, 4, 3))).astype(np.float32)
    F64 = F.astype(np.longdouble)
    hi = 3

    def S(p):
        v = np.zeros(3, dtype=np.longdouble)
        for k in range(4):
            for j in range(4):
                for i in range(4):
                    w = (max(0, 1 - abs(p[0] - i)) * max(0, 1 - abs(p[1] - j)) * max(0, 1 - abs(p[2] - k)))
                    v += w * F64[k, j, i]
        return v

    def inside(q):
        return all(0 <= x <= hi for x in q)

    dt = np.longdouble(0.3)
    seeds = rng.uniform(0.2, 2.8, size=(6, 3))
    L = oracle.trace_streamlines(F, (0, 0, 0), (1, 1, 1), seeds, dt=float(dt), max_steps=12, eps=0.0)
    for s in range(len(seeds)):
        p = seeds[s].astype(np.longdouble)
        verts = [p.copy()]
        status = oracle.MAXSTEPS
        for _ in range(12):
            k1 = dt * S(p)
            q = p + k1 / 2
            if not inside(q):
                status = oracle.EXIT
                break
            k2 = dt * S(q)
            q = p + k2 / 2
            if not inside(q):
                status = oracle.EXIT
                break
            k3 = dt * S(q)
            q = p + k3
            if not inside(q):
                status = oracle.EXIT
                break
            k4 = dt * S(q)
            pn = p + (k1 + 2 * k2 + 2 * k3 + k4) / 6
            if not inside(pn):
                status = oracle.EXIT
                break
            p = pn
            verts.append(p.copy())
        assert L.status[s] == status
        assert L.length[s] == len(verts)
        np.testing.assert_allclose(L.line(s), np.array(verts, dtype=np.float64), atol=1e-12)


# ---------------------------------------------------------------- termination rules

def test_zero_field_stops_stagnant_at_step0():
    g = unit_grid(8)
    F = np.zeros((8, 8, 8, 3), np.float32)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, np.array([[3.0, 3.0, 3.0]]), dt=0.1, max_steps=10)
    assert L.status[0] == oracle.STAGNANT and L.length[0] == 1 and L.margin[0] == 1.0


def test_eps_threshold_is_world_speed_before_the_step():
    g = inputs.Grid((8, 8, 8), (0, 0, 0), (0.5, 0.5, 0.5))
    F = inputs.uniform_field(g, (3e-7, 0.0, 4e-7))       # |v| = 5e-7 world units
    s = np.array([[1.0, 1.0, 1.0]])
    a = oracle.trace_streamlines(F, g.origin, g.spacing, s, dt=0.1, max_steps=3, eps=1e-6)
    b = oracle.trace_streamlines(F, g.origin, g.spacing, s, dt=0.1, max_steps=3, eps=4e-7)
    assert a.status[0] == oracle.STAGNANT and a.length[0] == 1
    assert abs(a.margin[0] - 0.5) < 1e-6
    assert b.status[0] == oracle.MAXSTEPS and b.length[0] == 4


def test_nan_in_field_stops_nanfield():
    g = unit_grid(8)
    F = inputs.uniform_field(g, (1.0, 0.0, 0.0))
    F[3, 3, 5, 0] = np.nan
    L = oracle.trace_streamlines(F, g.origin, g.spacing, np.array([[1.0, 3.0, 3.0]]), dt=0.5, max_steps=20)
    assert L.status[0] == oracle.NANFIELD
    # samples touch x=5 once a stage point passes x=4
    assert np.all(L.line(0)[:, 0] <= 4.0)


def test_max_steps_zero_and_one_and_outside_seed():
    g = unit_grid(8)
    F = inputs.uniform_field(g, (0.25, 0.0, 0.0))
    seeds = np.array([[1.0, 1.0, 1.0], [7.5, 1.0, 1.0], [-0.001, 2, 2], [7.0, 7.0, 7.0]])
    L0 = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt=1.0, max_steps=0)
    L1 = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt=1.0, max_steps=1)
    assert list(L0.status) == [oracle.MAXSTEPS, oracle.OUT, oracle.OUT, oracle.MAXSTEPS]
    assert list(L0.length) == [1, 0, 0, 1]
    assert list(L1.status) == [oracle.MAXSTEPS, oracle.OUT, oracle.OUT, oracle.EXIT]
    assert list(L1.length) == [2, 0, 0, 1]
    np.testing.assert_array_equal(L1.line(0), [[1, 1, 1], [1.25, 1, 1]])


def test_upper_face_sample_uses_clamped_cell():
    rng = np.random.default_rng(2)
    F = rng.standard_normal((5, 5, 5, 3)).astype(np.float32)
    v = oracle.sample(F, np.array([[4.0, 4.0, 4.0], [4.0, 2.0, 0.0]]))
    np.testing.assert_allclose(v[0], F[4, 4, 4], rtol=0, atol=1e-12)
    np.testing.assert_allclose(v[1], F[0, 2, 4], rtol=0, atol=1e-12)


def test_empty_seed_set():
    g = unit_grid(4)
    F = np.zeros((4, 4, 4, 3), np.float32)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, np.zeros((0, 3)), dt=0.1, max_steps=5)
    assert L.length.shape == (0,)


# ---------------------------------------------------------------- bricks

def test_brick_cells_and_ownership():
    assert oracle.brick_cells((512, 512, 512), (4, 4, 4)) == (128, 128, 128)
    assert oracle.brick_cells((64, 64, 64), (1, 1, 1)) == (63, 63, 63)
    assert oracle.brick_cells((1024, 1024, 1024), (4, 4, 4)) == (256, 256, 256)
    assert oracle.brick_cells((9, 17, 5), (2, 3, 4)) == (4, 6, 1)
    with pytest.raises(ValueError):
        oracle.brick_cells((4, 4, 4), (4, 1, 1))        # last brick would own no cell
    d, b = (512, 512, 512), (4, 4, 4)
    assert oracle.owner_brick(d, b, (128.0, 0.0, 383.999)) == (1, 0, 2)    # interior face -> upper
    assert oracle.owner_brick(d, b, (511.0, 384.0, 127.99999)) == (3, 3, 0)
    assert oracle.owner_brick(d, b, (0.0, 255.5, 256.0)) == (0, 1, 2)


# ---------------------------------------------------------------- quantisation

def _pow2_ceil(m):
    if m <= 0:
        return 1.0
    fr, e = np.frexp(np.float32(m))
    return float(np.float32(m)) if fr == 0.5 else float(2.0 ** int(e))


@pytest.mark.parametrize("dtype", [oracle.BF16, oracle.F16])
def test_quantized_codes_match_library_conversions(dtype):
    g = inputs.cube_grid(9)
    F = inputs.abc_field(g) * np.float32(3.0)
    F[2, 3, 4, 1] = np.nan
    F[0, 0, 0, 2] = np.float32(1e-9)          # FP16 subnormal after scaling
    bricks = (2, 2, 1)
    scales, codes, deq = oracle.quantize_field(F, bricks, dtype, want_codes=True)
    n = oracle.brick_cells((9, 9, 9), bricks)
    for bz in range(bricks[2]):
        for by in range(bricks[1]):
            for bx in range(bricks[0]):
                b = (bz * bricks[1] + by) * bricks[0] + bx
                ix = np.clip(bx * n[0] - 1 + np.arange(n[0] + 3), 0, 8)
                iy = np.clip(by * n[1] - 1 + np.arange(n[1] + 3), 0, 8)
                iz = np.clip(bz * n[2] - 1 + np.arange(n[2] + 3), 0, 8)
                stored = F[np.ix_(iz, iy, ix)]
                fin = stored[np.isfinite(stored)]
                assert scales[b] == _pow2_ceil(np.abs(fin).max())
                r = (stored / np.float32(scales[b])).astype(np.float32)
                if dtype == oracle.BF16:
                    ref = torch.from_numpy(r.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
                else:
                    ref = r.astype(np.float16).view(np.uint16)
                got = codes[b]
                fin_mask = np.isfinite(r)
                np.testing.assert_array_equal(got[fin_mask], ref[fin_mask])
                assert np.all((got[~fin_mask] & 0x7FFF) > (0x7F80 if dtype == oracle.BF16 else 0x7C00))


@pytest.mark.parametrize("dtype,bound", [(oracle.BF16, 2.0 ** -9), (oracle.F16, 2.0 ** -12)])
def test_quantization_error_bound_and_brick_independence(dtype, bound):
    g = inputs.cube_grid(17)
    modes = inputs.turbulence_modes(3, n_modes=16, kmax=4)
    F = inputs.turbulence_field(g, modes).numpy()
    bricks = (2, 2, 2)
    scales, codes, deq = oracle.quantize_field(F, bricks, dtype, want_codes=True)
    n = oracle.brick_cells((17, 17, 17), bricks)
    # decode(encode(v)) within half an ulp of the scaled format
    for b in range(8):
        bx, by, bz = b % 2, (b // 2) % 2, b // 4
        ix = np.clip(bx * n[0] - 1 + np.arange(n[0] + 3), 0, 16)
        iy = np.clip(by * n[1] - 1 + np.arange(n[1] + 3), 0, 16)
        iz = np.clip(bz * n[2] - 1 + np.arange(n[2] + 3), 0, 16)
        stored = F[np.ix_(iz, iy, ix)].astype(np.float64)
        dec = np.vectorize(lambda c: oracle.decode(int(c), float(scales[b]), dtype))(codes[b])
        assert np.abs(dec - stored).max() <= scales[b] * bound
        # a power-of-two scale makes the decode independent of the brick (away from subnormals)
        big = np.abs(stored) > scales[b] * 2.0 ** -13
        ref = deq[np.ix_(iz, iy, ix)].astype(np.float64)
        np.testing.assert_array_equal(dec[big], ref[big])


# ---------------------------------------------------------------- streaklines

def test_streaklines_in_steady_field_follow_streamline_vertices():
    n = 32
    g = unit_grid(n)
    c = (n - 1) / 2.0
    F = inputs.rotation_field(g, center=(c, c, c))
    nsl, steps, inj = 6, 5, 4
    slices = np.stack([F] * nsl)
    release = np.array([[20.0, 15.5, 3.0], [10.25, 18.0, 30.0]])
    dt = 0.07
    S = oracle.trace_streaklines(slices, g.origin, g.spacing, 1.0 * dt, release, dt, steps, inj)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, release, dt, steps)
    for r in range(2):
        for b in range(inj):
            assert S.status[r, b] == oracle.ACTIVE
            assert S.steps[r, b] == steps - b
            np.testing.assert_allclose(S.pos[r, b], L.line(r)[steps - b], atol=1e-12)


def test_streakline_time_interpolation_is_exact_for_linear_in_time_flow():
    n = 64
    g = unit_grid(n)
    a = np.array([0.5, 0.25, 0.0])
    bvel = np.array([1.0, -0.5, 0.75])
    F0 = inputs.uniform_field(g, a)
    F1 = inputs.uniform_field(g, bvel)
    slices = np.stack([F0, F1, F1, F1])
    dt = 0.25
    sdt = 0.5                                   # two steps per slice interval
    steps, inj = 5, 3
    x0 = np.array([[10.0, 40.0, 5.0]])
    S = oracle.trace_streaklines(slices, g.origin, g.spacing, sdt, x0, dt, steps, inj)

    def exact(t0, t1):
        # x(t1) - x(t0) for v(t) = a + (b-a) t/sdt on [0, sdt], b afterwards
        def X(t):
            if t <= sdt:
                return a * t + (bvel - a) * t * t / (2 * sdt)
            return X(sdt) + bvel * (t - sdt)
        return X(t1) - X(t0)

    for b in range(inj):
        expect = x0[0] + exact(b * dt, steps * dt)
        np.testing.assert_allclose(S.pos[0, b], expect, atol=1e-13)
        assert S.steps[0, b] == steps - b


def test_max_speed_planted_pythagorean_samples():
    # The speed in cells per unit time of a sample v on spacing s is |v / s|.
    # Samples are planted whose velocity in cells is a Pythagorean quadruple,
    # so the expected maximum is an integer fixed by arithmetic alone: (1, 4, 8)
    # has norm 9, (2, 3, 6) norm 7.  The spacing differs per axis, so dividing
    # by the wrong axis, dropping a component or skipping the division changes
    # the answer; planting at the last sample catches a loop that stops early.
    sp = (0.5, 0.25, 2.0)
    g = inputs.Grid((5, 6, 7), (0.0, 1.0, 2.0), sp)
    rng = np.random.default_rng(5)
    F = (0.01 * rng.uniform(-1, 1, (7, 6, 5, 3))).astype(np.float32)   # background: under 0.2 cells/time
    assert oracle.max_speed(F, g.spacing) < 0.2

    def plant(F, z, y, x, cells):
        F[z, y, x] = [cells[a] * sp[a] for a in range(3)]              # exact in float32 (dyadic)

    plant(F, 2, 3, 1, (2, 3, 6))
    assert oracle.max_speed(F, g.spacing) == 7.0
    plant(F, 6, 5, 4, (1, 4, 8))                                        # the very last sample
    assert oracle.max_speed(F, g.spacing) == 9.0
    # the same components permuted across axes: the grid's anisotropy changes |v/s|
    F2 = F.copy()
    F2[6, 5, 4] = [8 * sp[0], 1 * sp[1], 4 * sp[2]]
    assert oracle.max_speed(F2, g.spacing) == 9.0
    F3 = F.copy()
    F3[6, 5, 4] = [1 * sp[2], 4 * sp[1], 8 * sp[0]]                     # cells (4, 4, 2): speed 6
    assert oracle.max_speed(F3, g.spacing) == 7.0                       # the (2, 3, 6) sample is now the largest
    # negative components count by magnitude
    F4 = F.copy()
    F4[0, 0, 0] = [-2 * sp[0], -10 * sp[1], 11 * sp[2]]                 # (2, 10, 11): 15
    assert oracle.max_speed(F4, g.spacing) == 15.0


def test_max_speed_uniform_and_rotation_closed_forms():
    # uniform flow u: every sample has speed |u / s|; (3 * 0.5, 4 * 0.25, 12 * 2.0) -> (3, 4, 12): 13
    sp = (0.5, 0.25, 2.0)
    g = inputs.Grid((4, 5, 6), (1.0, -2.0, 0.5), sp)
    F = inputs.uniform_field(g, (1.5, 1.0, 24.0))
    assert oracle.max_speed(F, g.spacing) == 13.0
    # solid-body rotation v = (-(y - cy), x - cx, 0) on a unit-spacing grid with
    # the axis at the centre: the largest speed is at a corner, the distance
    # from the axis sqrt(hx^2 + hy^2) with hx, hy the half extents
    g2 = inputs.Grid((9, 7, 3), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    F2 = inputs.rotation_field(g2, center=(4.0, 3.0, 1.0))
    assert oracle.max_speed(F2, g2.spacing) == 5.0                      # (4, 3) -> 5


def test_golden_uniform_exit():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "uniform_exit.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for r in rows:
        sx, sy, sz, dt, nv, st, mg = map(float, r)
        g = unit_grid(17)
        F = inputs.uniform_field(g, (1.0, 0.0, 0.0))
        L = oracle.trace_streamlines(F, g.origin, g.spacing, np.array([[sx, sy, sz]]), dt=dt, max_steps=1000)
        assert L.length[0] == int(nv) and L.status[0] == int(st) and L.margin[0] == mg


def test_fx21_codes_match_numpy_rounding_and_error_bound():
    g = inputs.cube_grid(13)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(6, n_modes=16, kmax=3)).numpy() * np.float32(5.0)
    F[1, 2, 3, 0] = np.inf
    bricks = (2, 1, 2)
    scales, codes, deq = oracle.quantize_field(F, bricks, oracle.FX21, want_codes=True)
    n = oracle.brick_cells(g.dims, bricks)
    for b in range(4):
        bx, bz = b % 2, b // 2
        ix = np.clip(bx * n[0] - 1 + np.arange(n[0] + 3), 0, 12)
        iy = np.clip(-1 + np.arange(n[1] + 3), 0, 12)
        iz = np.clip(bz * n[2] - 1 + np.arange(n[2] + 3), 0, 12)
        stored = F[np.ix_(iz, iy, ix)]
        fin = np.isfinite(stored).all(axis=-1)
        s_b = _pow2_ceil(np.abs(stored[np.isfinite(stored)]).max())
        assert scales[b] == np.float32(s_b / 2 ** 20)          # the quantum
        # numpy's rint rounds half to even
        ref = np.clip(np.rint((stored / np.float32(s_b)).astype(np.float64) * 2 ** 20), -(2 ** 20 - 1), 2 ** 20 - 1)
        np.testing.assert_array_equal(codes[b][fin], ref[fin].astype(np.int32))
        assert (codes[b][~fin] == np.iinfo(np.int32).min).all()
        err = np.abs(codes[b][fin].astype(np.float64) * scales[b] - stored[fin])
        assert err.max() <= s_b * 2.0 ** -21
    assert np.isnan(deq[1, 2, 3]).all()


# ---------------------------------------------------------------- backward integration

def test_backward_uniform_flow_exact_line_and_exit():
    # backward lines follow -v: the uniform-flow line runs to the lower face
    g = unit_grid(17)
    F = inputs.uniform_field(g, (1.0, 0.0, 0.0))
    seed = np.array([[9.0, 5.5, 7.25]])
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seed, dt=-0.25, max_steps=500)
    # p_n = 9 - n/4; the step from x = 0 has its first stage point at -0.125 < 0
    assert L.status[0] == oracle.EXIT
    assert L.length[0] == 37
    np.testing.assert_array_equal(L.line(0)[:, 0], 9.0 - 0.25 * np.arange(37))
    assert L.margin[0] == 0.125


def test_backward_is_forward_in_the_negated_field():
    # RK4 with -dt on v takes exactly the steps of RK4 with dt on -v (every
    # stage is dt * v(P) and negation is exact), so the lines agree bit for bit
    g = inputs.cube_grid(21)
    F = inputs.turbulence_field(g, inputs.turbulence_modes(31, n_modes=24, kmax=3)).numpy()
    seeds = inputs.uniform_seeds(g, 200, 31)
    dt = 0.5 / oracle.max_speed(F, g.spacing)
    a = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, -dt, 300)
    b = oracle.trace_streamlines(-F, g.origin, g.spacing, seeds, dt, 300)
    np.testing.assert_array_equal(a.length, b.length)
    np.testing.assert_array_equal(a.status, b.status)
    np.testing.assert_array_equal(a.verts, b.verts)
    # and a backward step undoes a forward one to RK4's local error (h^5)
    org, sp = np.asarray(g.origin), np.asarray(g.spacing)
    f = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 1)
    ok = np.flatnonzero(f.length == 2)
    ends = np.stack([org + sp * f.line(i)[1] for i in ok])
    back = oracle.trace_streamlines(F, g.origin, g.spacing, ends, -dt, 1)
    assert (back.length == 2).all()
    ret = np.stack([back.line(i)[1] for i in range(len(ok))])          # index space
    start = (seeds[ok].astype(np.float64) - org) / sp
    err = np.abs(ret - start).max()
    assert 0 < err < 1e-3           # h = 0.5 cell: (h)^5 scale, far below a cell, yet not exact


# ---------------------------------------------------------------- path lines

def test_pathlines_in_steady_field_are_streamlines():
    n = 32
    g = unit_grid(n)
    c = (n - 1) / 2.0
    F = inputs.rotation_field(g, center=(c, c, c))
    slices = np.stack([F] * 5)
    seeds = np.array([[20.0, 15.5, 3.0], [10.25, 18.0, 30.0], [-1.0, 2.0, 2.0]])
    dt = 0.07
    P = oracle.trace_pathlines(slices, g.origin, g.spacing, 3 * dt, seeds, dt, 40)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 40)
    np.testing.assert_array_equal(P.length, L.length)
    np.testing.assert_array_equal(P.status, L.status)
    for i in range(3):
        np.testing.assert_allclose(P.line(i), L.line(i), atol=1e-12)


def test_pathlines_exact_for_linear_in_time_flow():
    # v(t) = a + (b - a) t / sdt on [0, sdt], b afterwards, the same at every
    # point: RK4 integrates a polynomial of degree <= 3 in t exactly, so the
    # vertices are the closed-form trajectory to rounding
    n = 64
    g = unit_grid(n)
    a = np.array([0.5, 0.25, 0.0])
    bvel = np.array([1.0, -0.5, 0.75])
    slices = np.stack([inputs.uniform_field(g, a), inputs.uniform_field(g, bvel), inputs.uniform_field(g, bvel)])
    dt, sdt = 0.25, 0.5
    x0 = np.array([[10.0, 40.0, 5.0]])
    P = oracle.trace_pathlines(slices, g.origin, g.spacing, sdt, x0, dt, 12)
    assert P.status[0] == oracle.MAXSTEPS and P.length[0] == 13

    def X(t):
        if t <= sdt:
            return a * t + (bvel - a) * t * t / (2 * sdt)
        return X(sdt) + bvel * (t - sdt)

    for j in range(13):
        np.testing.assert_allclose(P.line(0)[j], x0[0] + X(j * dt), atol=1e-12)


# ---------------------------------------------------------------- unstructured fields

_A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.1]])
_B = np.array([0.5, -0.25, 0.75])


@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_umesh_cells_reproduce_linear_fields(kind):
    # every isoparametric cell reproduces a field linear in x exactly, whatever
    # the shape of the (jittered) cell: a check of point location, Newton's
    # inversion and the shape functions together
    g = inputs.Grid((6, 5, 4), (1.0, -2.0, 0.5), (0.5, 0.75, 1.0))
    m = inputs.grid_mesh(g, np.zeros((4, 5, 6, 3)), kind=kind, jitter=0.25, seed=7)
    m["velocity"] = m["vertices"] @ _A.T + _B
    lo = np.asarray(g.origin) + 0.01
    hi = np.asarray(g.origin) + np.asarray(g.spacing) * (np.asarray(g.dims) - 1) - 0.01
    pts = lo + (hi - lo) * inputs.uniform(5, 1, 3000).reshape(-1, 3)
    v, cell = oracle.umesh_sample(m, pts)
    assert (cell >= 0).all()
    np.testing.assert_allclose(v, pts @ _A.T + _B, atol=1e-12)
    out = np.array([[lo[0] - 0.5, lo[1] + 1, lo[2] + 1], [hi[0] + 0.3, lo[1], lo[2]], [lo[0], lo[1], hi[2] + 2.0]])
    _, c = oracle.umesh_sample(m, out)
    assert (c == -1).all()


def test_umesh_hexes_of_a_grid_trace_the_structured_lines():
    # undistorted hexahedra of a grid interpolate trilinearly in the grid's
    # fractions: the unstructured field is the structured one
    g = inputs.Grid((13, 11, 12), (0.5, -1.0, 2.0), (0.5, 0.25, 0.75))
    F = inputs.turbulence_field(g, inputs.turbulence_modes(8, n_modes=24, kmax=2)).numpy()
    m = inputs.grid_mesh(g, F, kind="hex")
    seeds = inputs.uniform_seeds(g, 60, 8)
    dt = 0.4 / oracle.max_speed(F, g.spacing)
    L = oracle.trace_streamlines(F, g.origin, g.spacing, seeds, dt, 80)
    U = oracle.trace_umesh(m, seeds, dt, 80)
    org, sp = np.asarray(g.origin), np.asarray(g.spacing)
    for i in range(len(seeds)):
        if L.status[i] == oracle.EXIT and abs(L.length[i] - U.length[i]) <= 1:
            continue                                     # a stage point on the boundary face
        assert L.length[i] == U.length[i] and L.status[i] == U.status[i]
        np.testing.assert_allclose(U.line(i), org + sp * L.line(i), atol=1e-9)


def test_umesh_uniform_flow_exact_line_and_exit():
    g = inputs.Grid((9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    m = inputs.grid_mesh(g, inputs.uniform_field(g, (0.25, 0.0, 0.0)), kind="tet", jitter=0.2, seed=2)
    seed = np.array([[1.0, 4.3, 3.7]])
    U = oracle.trace_umesh(m, seed, 1.0, 100)
    # p_n = 1 + n/4 along x; the step from x = 8 has its first stage point at 8.125
    assert U.status[0] == oracle.EXIT and U.length[0] == 29
    np.testing.assert_allclose(U.line(0)[:, 0], 1.0 + 0.25 * np.arange(29), atol=1e-12)
