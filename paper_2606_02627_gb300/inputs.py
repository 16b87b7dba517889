"""Seeded synthetic inputs: counter-based random numbers, vector fields and seeds.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds no arithmetic of the advection method itself (no
sampling, no integration, no quantisation); it only makes input arrays.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value i of stream s under seed k is mix64(key(k, s) + (i + 1) * G),
with G the golden-ratio increment 0x9E3779B97F4A7C15.  Uniform doubles take
the top 53 bits.

The field and seed recipes stand in for the paper's datasets (MHD turbulence,
the 1K^3 galaxy and the wind farm of Sec. 4 and Sec. 5), which are not
available here:

* ``turbulence``: a divergence-free sum of random Fourier modes on [0, 2pi]^3
  with |k|^(-5/3) amplitudes and random phases.
* ``rotation`` / ``abc`` / ``uniform`` / ``linear``: analytic fields whose
  trajectories have closed forms.

Grid arrays are AoS ``[nz][ny][nx][3]`` float32 (x fastest), world units.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
TWO_PI = 2.0 * math.pi


def _mix64_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> int:
    """Key of stream ``stream`` under ``seed`` (independent sub-sequences)."""
    return _mix64_int((seed * GAMMA + 0x632BE59BD9B4E019 * (stream + 1)) & MASK64)


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Counter-based SplitMix64 outputs ``start .. start+count-1`` as uint64."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + idx * np.uint64(GAMMA)
    return _mix64_np(z)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each output."""
    return (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of pairs of uniforms."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]          # (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(TWO_PI * u2)


# --------------------------------------------------------------------------
# grids


@dataclass(frozen=True)
class Grid:
    """A uniform grid of samples at world = origin + spacing * index."""
    dims: tuple            # (nx, ny, nz) samples per axis
    origin: tuple          # world position of sample (0, 0, 0)
    spacing: tuple         # world distance between samples per axis

    def world_axes(self):
        return [self.origin[a] + self.spacing[a] * np.arange(self.dims[a], dtype=np.float64)
                for a in range(3)]


def cube_grid(n: int, lo: float = 0.0, hi: float = TWO_PI) -> Grid:
    """n^3 samples on the closed box [lo, hi]^3 (inclusive: spacing (hi-lo)/(n-1))."""
    h = (hi - lo) / (n - 1)
    return Grid((n, n, n), (lo, lo, lo), (h, h, h))


def _eval_on_grid(grid: Grid, fn) -> np.ndarray:
    x, y, z = grid.world_axes()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    vx, vy, vz = fn(X, Y, Z)
    out = np.empty(tuple(reversed(grid.dims)) + (3,), dtype=np.float64)
    out[..., 0] = vx
    out[..., 1] = vy
    out[..., 2] = vz
    return out


def rotation_field(grid: Grid, center=(math.pi, math.pi, math.pi), omega: float = 1.0,
                   dtype=np.float32) -> np.ndarray:
    """Solid-body rotation about the z axis through ``center``: v = omega(-(y-cy), x-cx, 0)."""
    cx, cy, _ = center
    return _eval_on_grid(grid, lambda X, Y, Z: (-omega * (Y - cy), omega * (X - cx), 0.0 * Z)).astype(dtype)


ABC_A, ABC_B, ABC_C = math.sqrt(3.0), math.sqrt(2.0), 1.0


def abc_value(x, y, z, A=ABC_A, B=ABC_B, C=ABC_C):
    """Arnold-Beltrami-Childress flow (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)."""
    return (A * np.sin(z) + C * np.cos(y), B * np.sin(x) + A * np.cos(z), C * np.sin(y) + B * np.cos(x))


def abc_field(grid: Grid, dtype=np.float32) -> np.ndarray:
    return _eval_on_grid(grid, abc_value).astype(dtype)


def uniform_field(grid: Grid, u=(1.0, 0.0, 0.0), dtype=np.float32) -> np.ndarray:
    out = np.empty(tuple(reversed(grid.dims)) + (3,), dtype=dtype)
    out[...] = np.asarray(u, dtype=dtype)
    return out


def linear_field(grid: Grid, A, b, dtype=np.float32) -> np.ndarray:
    """v(x) = A x + b in world units."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return _eval_on_grid(grid, lambda X, Y, Z: tuple(A[r, 0] * X + A[r, 1] * Y + A[r, 2] * Z + b[r]
                                                   for r in range(3))).astype(dtype)


# --------------------------------------------------------------------------
# synthetic turbulence


@dataclass(frozen=True)
class Modes:
    k: np.ndarray        # (M, 3) integer wave vectors, 1 <= |k| <= kmax
    amp: np.ndarray      # (M,) |k|^(-5/3)
    xi: np.ndarray       # (M, 3) unit polarisation, perpendicular to k
    phase: np.ndarray    # (M,) in [0, 2 pi)
    rate: np.ndarray     # (M,) phase advance rate c_m in [0.5, 1.5] (unsteady fields)


def turbulence_modes(seed: int, n_modes: int = 256, kmax: int = 16, slope: float = -5.0 / 3.0) -> Modes:
    """Random Fourier modes: k uniform over integer vectors with 1 <= |k| <= kmax.

    k is drawn by rejection from the cube [-kmax, kmax]^3; the polarisation is
    xi = normalize(k x r) with r Gaussian, so every mode (and the sum) is
    divergence-free; amplitudes are |k|^slope (slope -5/3 taken literally).
    """
    ks = []
    i = 0
    side = 2 * kmax + 1
    while len(ks) < n_modes:
        u = uniform(seed, 0, 3 * 64, start=3 * 64 * i)
        i += 1
        c = np.floor(u * side).astype(np.int64) - kmax
        for t in range(64):
            kv = c[3 * t:3 * t + 3]
            n2 = int(kv @ kv)
            if 1 <= n2 <= kmax * kmax:
                ks.append(kv.copy())
                if len(ks) == n_modes:
                    break
    k = np.array(ks, dtype=np.int64)
    r = gaussian(seed, 1, 3 * n_modes).reshape(n_modes, 3)
    xi = np.cross(k.astype(np.float64), r)
    xi /= np.linalg.norm(xi, axis=1, keepdims=True)
    amp = np.linalg.norm(k.astype(np.float64), axis=1) ** slope
    phase = TWO_PI * uniform(seed, 2, n_modes)
    rate = 0.5 + uniform(seed, 3, n_modes)
    return Modes(k, amp, xi, phase, rate)


def turbulence_value(modes: Modes, x, y, z, time_slice: float = 0.0, n_slices: int = 64):
    """Direct FP64 evaluation of the mode sum at world points (for spot checks)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros(x.shape + (3,), dtype=np.float64)
    ph = modes.phase + TWO_PI * modes.rate * time_slice / n_slices
    for m in range(len(modes.amp)):
        arg = modes.k[m, 0] * x + modes.k[m, 1] * y + modes.k[m, 2] * z + ph[m]
        c = modes.amp[m] * np.cos(arg)
        out += c[..., None] * modes.xi[m]
    return out


def turbulence_field(grid: Grid, modes: Modes, time_slice: float = 0.0, n_slices: int = 64,
                     device=None, out=None):
    """Mode sum on the grid, float32 AoS ``[nz][ny][nx][3]``.

    The phase factor of each mode is separable, exp(i k.x) = exp(i kx x)
    exp(i ky y) exp(i kz z); the 1-D factors are formed in FP64 and the 3-D
    product is taken plane by plane (complex64 on a CUDA device, complex128 on
    the CPU).  With ``device`` a torch device the result is a torch tensor on it.
    """
    import torch

    dev = torch.device(device) if device is not None else torch.device("cpu")
    cplx = torch.complex64 if dev.type == "cuda" else torch.complex128
    real = torch.float32 if dev.type == "cuda" else torch.float64
    nx, ny, nz = grid.dims
    xs, ys, zs = grid.world_axes()
    ph = modes.phase + TWO_PI * modes.rate * time_slice / n_slices
    if out is None:
        out = torch.zeros((nz, ny, nx, 3), dtype=torch.float32, device=dev)
    else:
        out.zero_()
    M = len(modes.amp)
    ex = np.exp(1j * np.outer(modes.k[:, 0], xs))                      # (M, nx)
    ey = np.exp(1j * np.outer(modes.k[:, 1], ys))                      # (M, ny)
    ez = np.exp(1j * (np.outer(modes.k[:, 2], zs) + ph[:, None]))      # (M, nz)
    coef = torch.as_tensor(modes.amp[:, None] * modes.xi, dtype=real, device=dev)   # (M, 3)
    ex_t = torch.as_tensor(ex, dtype=cplx, device=dev)
    ey_t = torch.as_tensor(ey, dtype=cplx, device=dev)
    ez_t = torch.as_tensor(ez, dtype=cplx, device=dev)
    zchunk = max(1, min(nz, (1 << 26) // max(1, nx * ny)))
    for z0 in range(0, nz, zchunk):
        z1 = min(nz, z0 + zchunk)
        acc = torch.zeros((z1 - z0, ny, nx, 3), dtype=real, device=dev)
        for m in range(M):
            pxy = ey_t[m][:, None] * ex_t[m][None, :]                  # (ny, nx)
            w = (ez_t[m, z0:z1][:, None, None] * pxy[None]).real       # (zc, ny, nx)
            acc.add_(w[..., None] * coef[m])
        out[z0:z1] = acc.to(torch.float32)
    return out


# --------------------------------------------------------------------------
# seeds


def uniform_seeds(grid: Grid, n: int, seed: int, lo_cells: float = 0.0, hi_cells=None,
                  stream: int = 7) -> np.ndarray:
    """n seeds uniform in index box [lo, hi]^3 (hi defaults to N-1-lo), as world float32 (n, 3)."""
    u = uniform(seed, stream, 3 * n).reshape(n, 3)
    out = np.empty((n, 3), dtype=np.float64)
    for a in range(3):
        hi = (grid.dims[a] - 1 - lo_cells) if hi_cells is None else hi_cells
        idx = lo_cells + (hi - lo_cells) * u[:, a]
        out[:, a] = grid.origin[a] + grid.spacing[a] * idx
    return out.astype(np.float32)


def box_seeds(grid: Grid, n: int, seed: int, lo_idx, hi_idx, stream: int = 8) -> np.ndarray:
    """n seeds uniform in the index box [lo_idx, hi_idx] (per axis), world float32."""
    u = uniform(seed, stream, 3 * n).reshape(n, 3)
    lo = np.asarray(lo_idx, dtype=np.float64)
    hi = np.asarray(hi_idx, dtype=np.float64)
    idx = lo + (hi - lo) * u
    org = np.asarray(grid.origin)
    sp = np.asarray(grid.spacing)
    return (org + sp * idx).astype(np.float32)


def rake_seeds(grid: Grid, n: int, a_idx, b_idx) -> np.ndarray:
    """n seeds evenly spaced on the index segment from a_idx to b_idx inclusive, world float32."""
    a = np.asarray(a_idx, dtype=np.float64)
    b = np.asarray(b_idx, dtype=np.float64)
    t = np.linspace(0.0, 1.0, n) if n > 1 else np.zeros(1)
    idx = a[None, :] + (b - a)[None, :] * t[:, None]
    org = np.asarray(grid.origin)
    sp = np.asarray(grid.spacing)
    return (org + sp * idx).astype(np.float32)


def max_speed_cells(field: np.ndarray, spacing) -> float:
    """max over samples of |v / spacing| (cells per unit time), FP64 on the host."""
    f = np.asarray(field, dtype=np.float64).reshape(-1, 3) / np.asarray(spacing, dtype=np.float64)
    return float(np.sqrt((f * f).sum(axis=1)).max())


# ---------------------------------------------------------------- unstructured meshes

# VTK cell types by vertex count: tetrahedron 4, pyramid 5, wedge (prism) 6, hexahedron 8
TET, PYRAMID, PRISM, HEX = 4, 5, 6, 8

# local corner numbering of a grid cell: corner k at (k & 1, k >> 1 & 1, k >> 2)
_HEX_ORDER = (0, 1, 3, 2, 4, 5, 7, 6)          # VTK hexahedron order of those corners
# six tetrahedra around the main diagonal (corners 0 and 7), the same in every cell
_TETS = ((0, 1, 3, 7), (0, 3, 2, 7), (0, 2, 6, 7), (0, 6, 4, 7), (0, 4, 5, 7), (0, 5, 1, 7))
# two wedges: bottom triangles (0,1,3) and (0,3,2), extruded in z
_PRISMS = ((0, 1, 3, 4, 5, 7), (0, 3, 2, 4, 7, 6))
# six faces as (VTK-ordered quad) bases of pyramids with apex at the centre
_FACES = ((0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5))


def grid_mesh(grid: Grid, field: np.ndarray, kind: str = "hex", jitter: float = 0.0, seed: int = 0) -> dict:
    """The cells of a structured grid as an unstructured mesh: each cell as one
    hexahedron, six tetrahedra, two prisms or six pyramids (apex at the cell
    centre, an extra vertex whose velocity is the mean of the eight corners).
    jitter moves every interior vertex by up to jitter cells per axis
    (uniform, SplitMix64 stream 30); the velocity stays at the vertices."""
    nx, ny, nz = grid.dims
    org = np.asarray(grid.origin, dtype=np.float64)
    sp = np.asarray(grid.spacing, dtype=np.float64)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = org + sp * np.stack([i, j, k], -1).reshape(-1, 3).astype(np.float64)
    V = np.asarray(field, dtype=np.float64).reshape(-1, 3).copy()
    if jitter > 0.0:
        u = uniform(seed, 30, X.size).reshape(-1, 3) * 2.0 - 1.0
        inner = ((i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1) & (k > 0) & (k < nz - 1)).reshape(-1)
        X[inner] += (jitter * sp) * u[inner]
    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    base = ((ck * ny + cj) * nx + ci).reshape(-1)
    corner_off = np.array([((c >> 2) * ny + ((c >> 1) & 1)) * nx + (c & 1) for c in range(8)])
    corners = base[:, None] + corner_off[None, :]          # [n_cells, 8] in local corner numbering
    if kind == "hex":
        cells = corners[:, list(_HEX_ORDER)]
        types = np.full(len(cells), HEX, np.uint8)
    elif kind == "tet":
        cells = np.concatenate([corners[:, list(t)] for t in _TETS])
        types = np.full(len(cells), TET, np.uint8)
    elif kind == "prism":
        cells = np.concatenate([corners[:, list(p)] for p in _PRISMS])
        types = np.full(len(cells), PRISM, np.uint8)
    elif kind == "pyramid":
        n0 = len(X)
        centre = X[corners].mean(axis=1)
        X = np.concatenate([X, centre])
        V = np.concatenate([V, V[corners].mean(axis=1)])
        apex = n0 + np.arange(len(corners))
        cells = np.concatenate([np.concatenate([corners[:, list(f)], apex[:, None]], 1) for f in _FACES])
        types = np.full(len(cells), PYRAMID, np.uint8)
    else:
        raise ValueError(kind)
    nv = types.astype(np.int64)
    off = np.concatenate([[0], np.cumsum(nv)])
    return {"vertices": X, "velocity": V, "cell_vertices": cells.reshape(-1).astype(np.int32), "cell_offsets": off,
            "cell_types": types}
