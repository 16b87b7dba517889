"""Checks of the seeded synthetic inputs (SplitMix64, turbulence, seeds)."""
import math

import numpy as np

from paper_2606_02627_gb300 import inputs


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (next(): state += 0x9E3779B97F4A7C15; return mix(state)).
    z = [inputs._mix64_int((i + 1) * inputs.GAMMA & inputs.MASK64) for i in range(3)]
    assert z == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    a = inputs.u64(1, 0, 0, 5)
    b = inputs.u64(1, 0, 2, 3)
    np.testing.assert_array_equal(a[2:], b)                      # counter-based
    assert not np.array_equal(inputs.u64(1, 1, 0, 5), a)         # streams differ


def test_uniform_and_gaussian_moments():
    u = inputs.uniform(3, 0, 200_000)
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005
    g = inputs.gaussian(3, 1, 200_000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01


def test_turbulence_modes_properties():
    m = inputs.turbulence_modes(1)
    kn = np.linalg.norm(m.k, axis=1)
    assert m.k.shape == (256, 3) and kn.min() >= 1 and kn.max() <= 16
    np.testing.assert_allclose(m.amp, kn ** (-5 / 3))
    np.testing.assert_allclose(np.einsum("mi,mi->m", m.k.astype(float), m.xi), 0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(m.xi, axis=1), 1, atol=1e-12)
    assert m.phase.min() >= 0 and m.phase.max() < 2 * math.pi
    assert m.rate.min() >= 0.5 and m.rate.max() < 1.5
    # deterministic
    np.testing.assert_array_equal(inputs.turbulence_modes(1).k, m.k)


def test_turbulence_grid_matches_direct_evaluation_and_is_divergence_free():
    n = 33
    g = inputs.cube_grid(n)
    m = inputs.turbulence_modes(2, n_modes=64, kmax=4)
    F = inputs.turbulence_field(g, m).numpy()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, size=(200, 3))
    xs, ys, zs = g.world_axes()
    direct = inputs.turbulence_value(m, xs[idx[:, 0]], ys[idx[:, 1]], zs[idx[:, 2]])
    got = F[idx[:, 2], idx[:, 1], idx[:, 0]]
    scale = np.abs(direct).max()
    assert np.abs(got - direct).max() < 2e-6 * scale
    # central-difference divergence is O(h^2) small compared with the gradient
    h = g.spacing[0]
    d = ((F[1:-1, 1:-1, 2:, 0] - F[1:-1, 1:-1, :-2, 0])
         + (F[1:-1, 2:, 1:-1, 1] - F[1:-1, :-2, 1:-1, 1])
         + (F[2:, 1:-1, 1:-1, 2] - F[:-2, 1:-1, 1:-1, 2])) / (2 * h)
    grad = np.abs(F[1:-1, 1:-1, 2:, 0] - F[1:-1, 1:-1, :-2, 0]).max() / (2 * h)
    assert np.abs(d).max() < 0.1 * grad


def test_unsteady_phases_advance():
    g = inputs.cube_grid(9)
    m = inputs.turbulence_modes(3, n_modes=8, kmax=3)
    a = inputs.turbulence_field(g, m, time_slice=0).numpy()
    b = inputs.turbulence_field(g, m, time_slice=64).numpy()
    # after 64 slices each phase has advanced by 2 pi c_m: a different field
    assert np.abs(a - b).max() > 1e-3
    direct = inputs.turbulence_value(m, 0.0, 0.0, 0.0, time_slice=5)
    c = inputs.turbulence_field(g, m, time_slice=5).numpy()[0, 0, 0]
    np.testing.assert_allclose(c, direct, atol=1e-6)


def test_seed_generators():
    g = inputs.cube_grid(64)
    s = inputs.uniform_seeds(g, 1024, 0, lo_cells=1.0)
    idx = (s.astype(np.float64) - np.array(g.origin)) / np.array(g.spacing)
    assert idx.min() >= 1 - 1e-4 and idx.max() <= 62 + 1e-4
    r = inputs.rake_seeds(g, 5, (1, 1, 1), (5, 1, 1))
    np.testing.assert_allclose((r[:, 0] - g.origin[0]) / g.spacing[0], [1, 2, 3, 4, 5], rtol=1e-5)
    b = inputs.box_seeds(g, 100, 4, (10, 10, 10), (20, 30, 40))
    bi = (b.astype(np.float64) - np.array(g.origin)) / np.array(g.spacing)
    assert (bi >= np.array([10, 10, 10]) - 1e-4).all() and (bi <= np.array([20, 30, 40]) + 1e-4).all()
