"""ctypes wrapper of the FP64 C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg, never by the library.

The shared object is compiled with gcc on first use (or by ``build()``) into
this directory; ``-ffp-contract=off`` keeps the arithmetic the same on x86-64
and aarch64 hosts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

# line status values (the library's public header spells out the same numbers)
ACTIVE, MAXSTEPS, EXIT, STAGNANT, NANFIELD, OUT = 0, 1, 2, 3, 4, 5
NOT_RELEASED = 255
# storage types
F32, BF16, F16, FX21 = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than oracle.c."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            lib.or_trace_streamlines.argtypes = [P, P, P, P, P, i64, d, i64, d, P, P, P, P, ctypes.c_int]
            lib.or_trace_streamlines.restype = ctypes.c_int
            lib.or_trace_abc.argtypes = [d, d, d, P, P, P, P, i64, d, i64, d, P, P, P, P]
            lib.or_trace_abc.restype = ctypes.c_int
            lib.or_sample.argtypes = [P, P, P, i64, P]
            lib.or_sample.restype = ctypes.c_int
            lib.or_trace_streaklines.argtypes = [P, i64, P, P, P, d, P, i64, d, i64, i64, d, P, P, P, P,
                                                 ctypes.c_int]
            lib.or_trace_streaklines.restype = ctypes.c_int
            lib.or_trace_pathlines.argtypes = [P, i64, P, P, P, d, P, i64, d, i64, d, P, P, P, P, ctypes.c_int]
            lib.or_trace_pathlines.restype = ctypes.c_int
            lib.or_umesh_sample.argtypes = [P, P, P, P, P, i64, d, P, i64, P, P]
            lib.or_umesh_sample.restype = ctypes.c_int
            lib.or_umesh_trace.argtypes = [P, P, P, P, P, i64, i64, d, P, i64, d, i64, d, P, P, P, P, ctypes.c_int]
            lib.or_umesh_trace.restype = ctypes.c_int
            lib.or_brick_cells.argtypes = [P, P, P]
            lib.or_brick_cells.restype = ctypes.c_int
            lib.or_owner_brick.argtypes = [P, P, P, P]
            lib.or_owner_brick.restype = ctypes.c_int
            lib.or_quantize_field.argtypes = [P, P, P, ctypes.c_int, P, P, P]
            lib.or_quantize_field.restype = ctypes.c_int
            lib.or_decode.argtypes = [ctypes.c_uint16, ctypes.c_float, ctypes.c_int]
            lib.or_decode.restype = ctypes.c_double
            lib.or_max_speed.argtypes = [P, P, P]
            lib.or_max_speed.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _field(F):
    F = np.ascontiguousarray(F, dtype=np.float32)
    if F.ndim != 4 or F.shape[3] != 3:
        raise ValueError("field must be [nz][ny][nx][3]")
    dims = np.array([F.shape[2], F.shape[1], F.shape[0]], dtype=np.int64)
    return F, dims


class Lines:
    """Result of a streamline trace: per line a vertex list in index space."""

    def __init__(self, verts, length, status, margin):
        self.verts = verts          # (n, max_steps+1, 3) float64, index space
        self.length = length        # (n,) int32 vertex count
        self.status = status        # (n,) uint8
        self.margin = margin        # (n,) float64

    def line(self, i):
        return self.verts[i, : self.length[i]]

    def steps(self):
        return np.maximum(self.length.astype(np.int64) - 1, 0)


def trace_streamlines(F, origin, spacing, seeds_world, dt, max_steps, eps=1e-6, nthreads=0) -> Lines:
    """Steady RK4 streamlines on the trilinear field (FP64); see oracle.c."""
    lib = _load()
    F, dims = _field(F)
    seeds = np.ascontiguousarray(np.asarray(seeds_world, dtype=np.float64).reshape(-1, 3))
    n = seeds.shape[0]
    org = np.ascontiguousarray(origin, dtype=np.float64)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    verts = np.zeros((n, max_steps + 1, 3), dtype=np.float64)
    length = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.uint8)
    margin = np.zeros(n, dtype=np.float64)
    rc = lib.or_trace_streamlines(_p(F), _p(dims), _p(org), _p(sp), _p(seeds), n, float(dt),
                                  int(max_steps), float(eps), _p(verts), _p(length), _p(status),
                                  _p(margin), int(nthreads))
    if rc:
        raise ValueError("or_trace_streamlines: bad arguments")
    return Lines(verts, length, status, margin)


def trace_abc(dims, origin, spacing, seeds_world, dt, max_steps, eps=0.0, A=3 ** 0.5, B=2 ** 0.5, C=1.0):
    """RK4 on the analytic ABC flow (no grid), same loop as trace_streamlines."""
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    seeds = np.ascontiguousarray(np.asarray(seeds_world, dtype=np.float64).reshape(-1, 3))
    n = seeds.shape[0]
    org = np.ascontiguousarray(origin, dtype=np.float64)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    verts = np.zeros((n, max_steps + 1, 3), dtype=np.float64)
    length = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.uint8)
    margin = np.zeros(n, dtype=np.float64)
    lib.or_trace_abc(A, B, C, _p(dims), _p(org), _p(sp), _p(seeds), n, float(dt), int(max_steps),
                     float(eps), _p(verts), _p(length), _p(status), _p(margin))
    return Lines(verts, length, status, margin)


def sample(F, p_index):
    """Trilinear samples (world units) at index points (n, 3)."""
    lib = _load()
    F, dims = _field(F)
    p = np.ascontiguousarray(np.asarray(p_index, dtype=np.float64).reshape(-1, 3))
    v = np.zeros_like(p)
    lib.or_sample(_p(F), _p(dims), _p(p), p.shape[0], _p(v))
    return v


class Streaks:
    """Streakline particles, (R, n_inject) in release-major, birth-minor order."""

    def __init__(self, pos, status, steps, margin):
        self.pos = pos              # (R, n_inject, 3) index space
        self.status = status        # (R, n_inject) uint8
        self.steps = steps          # (R, n_inject) int32
        self.margin = margin


def trace_streaklines(slices, origin, spacing, slice_dt, release_world, dt, n_steps, n_inject,
                      eps=1e-6, nthreads=0) -> Streaks:
    lib = _load()
    S = np.ascontiguousarray(slices, dtype=np.float32)
    if S.ndim != 5 or S.shape[4] != 3:
        raise ValueError("slices must be [n_slices][nz][ny][nx][3]")
    dims = np.array([S.shape[3], S.shape[2], S.shape[1]], dtype=np.int64)
    rel = np.ascontiguousarray(np.asarray(release_world, dtype=np.float64).reshape(-1, 3))
    R = rel.shape[0]
    org = np.ascontiguousarray(origin, dtype=np.float64)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    pos = np.zeros((R, n_inject, 3), dtype=np.float64)
    status = np.zeros((R, n_inject), dtype=np.uint8)
    steps = np.zeros((R, n_inject), dtype=np.int32)
    margin = np.zeros((R, n_inject), dtype=np.float64)
    rc = lib.or_trace_streaklines(_p(S), S.shape[0], _p(dims), _p(org), _p(sp), float(slice_dt), _p(rel), R,
                                  float(dt), int(n_steps), int(n_inject), float(eps), _p(pos), _p(status),
                                  _p(steps), _p(margin), int(nthreads))
    if rc:
        raise ValueError("or_trace_streaklines: bad arguments")
    return Streaks(pos, status, steps, margin)


def trace_pathlines(slices, origin, spacing, slice_dt, seeds_world, dt, max_steps, eps=1e-6, nthreads=0) -> Lines:
    """Path lines through the slices (linear in time between them), FP64; see oracle.c."""
    lib = _load()
    S = np.ascontiguousarray(slices, dtype=np.float32)
    if S.ndim != 5 or S.shape[4] != 3:
        raise ValueError("slices must be [n_slices][nz][ny][nx][3]")
    dims = np.array([S.shape[3], S.shape[2], S.shape[1]], dtype=np.int64)
    seeds = np.ascontiguousarray(np.asarray(seeds_world, dtype=np.float64).reshape(-1, 3))
    n = seeds.shape[0]
    org = np.ascontiguousarray(origin, dtype=np.float64)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    verts = np.zeros((n, max_steps + 1, 3), dtype=np.float64)
    length = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.uint8)
    margin = np.zeros(n, dtype=np.float64)
    rc = lib.or_trace_pathlines(_p(S), S.shape[0], _p(dims), _p(org), _p(sp), float(slice_dt), _p(seeds), n,
                                float(dt), int(max_steps), float(eps), _p(verts), _p(length), _p(status),
                                _p(margin), int(nthreads))
    if rc:
        raise ValueError("or_trace_pathlines: bad arguments")
    return Lines(verts, length, status, margin)


def _umesh_args(mesh):
    X = np.ascontiguousarray(mesh["vertices"], dtype=np.float64).reshape(-1, 3)
    V = np.ascontiguousarray(mesh["velocity"], dtype=np.float64).reshape(-1, 3)
    idx = np.ascontiguousarray(mesh["cell_vertices"], dtype=np.int32)
    off = np.ascontiguousarray(mesh["cell_offsets"], dtype=np.int64)
    typ = np.ascontiguousarray(mesh["cell_types"], dtype=np.uint8)
    return X, V, idx, off, typ


def umesh_sample(mesh, points, tau=1e-6, nthreads=0):
    """Velocity (FP64) and containing cell (-1: none) at world points of an
    unstructured mesh (dict of vertices, velocity, cell_vertices, cell_offsets,
    cell_types); brute-force point location, see oracle.c."""
    lib = _load()
    X, V, idx, off, typ = _umesh_args(mesh)
    P = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    v = np.zeros_like(P)
    cell = np.zeros(len(P), dtype=np.int64)
    if lib.or_umesh_sample(_p(X), _p(V), _p(idx), _p(off), _p(typ), len(typ), float(tau), _p(P), len(P), _p(v),
                           _p(cell)):
        raise ValueError("or_umesh_sample: bad arguments")
    return v, cell


def trace_umesh(mesh, seeds_world, dt, max_steps, eps=1e-6, tau=1e-6, nthreads=0) -> Lines:
    """Streamlines on an unstructured mesh, FP64 (vertices in world coordinates)."""
    lib = _load()
    X, V, idx, off, typ = _umesh_args(mesh)
    seeds = np.ascontiguousarray(np.asarray(seeds_world, dtype=np.float64).reshape(-1, 3))
    n = seeds.shape[0]
    verts = np.zeros((n, max_steps + 1, 3), dtype=np.float64)
    length = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.uint8)
    margin = np.zeros(n, dtype=np.float64)
    rc = lib.or_umesh_trace(_p(X), _p(V), _p(idx), _p(off), _p(typ), len(typ), len(X), float(tau), _p(seeds), n,
                            float(dt),
                            int(max_steps), float(eps), _p(verts), _p(length), _p(status), _p(margin), int(nthreads))
    if rc:
        raise ValueError("or_umesh_trace: bad arguments")
    return Lines(verts, length, status, margin)


def brick_cells(dims, bricks):
    lib = _load()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    b = np.ascontiguousarray(bricks, dtype=np.int32)
    n = np.zeros(3, dtype=np.int64)
    if lib.or_brick_cells(_p(d), _p(b), _p(n)):
        raise ValueError("bad brick decomposition")
    return tuple(int(x) for x in n)


def owner_brick(dims, bricks, p_index):
    lib = _load()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    b = np.ascontiguousarray(bricks, dtype=np.int32)
    p = np.ascontiguousarray(p_index, dtype=np.float64)
    out = np.zeros(3, dtype=np.int32)
    if lib.or_owner_brick(_p(d), _p(b), _p(p), _p(out)):
        raise ValueError("bad brick decomposition")
    return tuple(int(x) for x in out)


def quantize_field(F, bricks, dtype, want_codes=False, want_dequant=True):
    """Per-brick scales, optional per-brick codes ((nb, S, S, S, 3) uint16, or int32
    for FX21) and the dequantised global field (float32, each sample with its
    owning brick's scale)."""
    lib = _load()
    F, dims = _field(F)
    b = np.ascontiguousarray(bricks, dtype=np.int32)
    n = brick_cells(dims, bricks)
    nb = int(b[0]) * int(b[1]) * int(b[2])
    scales = np.zeros(nb, dtype=np.float32)
    codes = None
    if want_codes and dtype != F32:
        codes = np.zeros((nb, n[2] + 3, n[1] + 3, n[0] + 3, 3), dtype=np.int32 if dtype == FX21 else np.uint16)
    deq = np.zeros_like(F) if want_dequant else None
    rc = lib.or_quantize_field(_p(F), _p(dims), _p(b), int(dtype), _p(scales),
                               _p(codes) if codes is not None else None,
                               _p(deq) if deq is not None else None)
    if rc:
        raise ValueError("or_quantize_field failed")
    return scales, codes, deq


def decode(code: int, scale: float, dtype: int) -> float:
    return _load().or_decode(int(code), float(scale), int(dtype))


def max_speed(F, spacing) -> float:
    lib = _load()
    F, dims = _field(F)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    return lib.or_max_speed(_p(F), _p(dims), _p(sp))


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
