"""Python objects over the C ABI: PyTorch provides device memory and streams.

Every step of the hot path runs in libstreamgb's kernels; this module only
allocates the caller-owned buffers the C ABI asks for and marshals pointers.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import call

DTYPES = {"f32": L.SG_F32, "bf16": L.SG_BF16, "f16": L.SG_F16, "fx21": L.SG_FX21}
LAYOUTS = {"linear": L.SG_LAYOUT_LINEAR, "tiled4": L.SG_LAYOUT_TILED4, "cell8": L.SG_LAYOUT_CELL8,
           "global": L.SG_FIELD_GLOBAL}
KERNELS = {"persistent": L.SG_KERNEL_PERSISTENT, "per_seed": L.SG_KERNEL_PER_SEED, "per_step": L.SG_KERNEL_PER_STEP,
           "lockstep": L.SG_KERNEL_LOCKSTEP}
DIRECTIONS = {"forward": L.SG_DIR_FORWARD, "backward": L.SG_DIR_BACKWARD, "both": L.SG_DIR_BOTH}
STATUS_NAMES = {0: "ACTIVE", 1: "MAXSTEPS", 2: "EXIT", 3: "STAGNANT", 4: "NANFIELD", 5: "OUT", 6: "HALO"}


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x) -> ctypes.c_void_p:
    if x is None:
        return ctypes.c_void_p(None)
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(int(x))


class Context:
    def __init__(self, device: int = 0):
        self.device = int(device)
        h = ctypes.c_void_p()
        call("sg_context_create", self.device, ctypes.byref(h))
        self.h = h
        n = ctypes.c_int32()
        call("sg_context_sm_count", self.h, ctypes.byref(n))
        self.sm_count = n.value

    def close(self):
        if self.h:
            L.lib().sg_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_desc(dims, origin, spacing, bricks=(1, 1, 1), dtype="f32", layout="linear", n_slots=1,
               slice_dt=1.0) -> L.sg_field_desc:
    d = L.sg_field_desc()
    for a in range(3):
        d.dims[a] = int(dims[a])
        d.origin[a] = float(origin[a])
        d.spacing[a] = float(spacing[a])
        d.bricks[a] = int(bricks[a])
    d.ghost = 1
    d.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    d.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    d.n_slots = int(n_slots)
    d.slice_dt = float(slice_dt)
    return d


class Field:
    """A bricked (or global float3) vector field in a torch-owned device buffer."""

    def __init__(self, ctx: Context, dims, origin, spacing, bricks=(1, 1, 1), dtype="f32", layout="linear",
                 n_slots=1, slice_dt=1.0):
        self.ctx = ctx
        self.desc = field_desc(dims, origin, spacing, bricks, dtype, layout, n_slots, slice_dt)
        nbytes = ctypes.c_size_t()
        call("sg_field_required_bytes", ctypes.byref(self.desc), ctypes.byref(nbytes))
        self.nbytes = nbytes.value
        self.storage = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=f"cuda:{ctx.device}")
        h = ctypes.c_void_p()
        call("sg_field_create", ctx.h, ctypes.byref(self.desc), _ptr(self.storage), self.nbytes, ctypes.byref(h))
        self.h = h
        self.dims = tuple(int(x) for x in dims)
        self.origin = tuple(float(x) for x in origin)
        self.spacing = tuple(float(x) for x in spacing)
        self.bricks = tuple(int(x) for x in bricks)
        self.dtype = dtype

    def brick_cells(self):
        n = (ctypes.c_int64 * 3)()
        call("sg_field_brick_cells", self.h, n)
        return tuple(n)

    def set_global(self, vec3, slot: int = 0, stream=None):
        """vec3: float32 [nz][ny][nx][3] on the device or in page-locked host memory."""
        assert vec3.dtype == torch.float32 and vec3.is_contiguous()
        call("sg_field_set_global", self.h, slot, _ptr(vec3), _stream(stream))

    def set_brick(self, bx, by, bz, vec3_with_halo, slot: int = 0, stream=None):
        assert vec3_with_halo.dtype == torch.float32 and vec3_with_halo.is_contiguous()
        call("sg_field_set_brick", self.h, slot, bx, by, bz, _ptr(vec3_with_halo), _stream(stream))

    def stream_slice(self, slice_index: int, pinned_host, stream=None):
        call("sg_field_stream_slice", self.h, slice_index, _ptr(pinned_host), _stream(stream))

    def max_speed(self, slot: int = 0, stream=None) -> float:
        v = ctypes.c_double()
        call("sg_field_max_speed", self.h, slot, ctypes.byref(v), _stream(stream))
        return v.value

    def read_brick(self, bx, by, bz, slot: int = 0, stream=None):
        n = self.brick_cells()
        shape = (n[2] + 3, n[1] + 3, n[0] + 3, 3)
        out = np.zeros(shape, dtype={L.SG_F32: np.float32, L.SG_FX21: np.int32}.get(self.desc.dtype, np.uint16))
        sc = ctypes.c_float()
        call("sg_field_read_brick", self.h, slot, bx, by, bz, _ptr(out), ctypes.byref(sc), _stream(stream))
        return out, sc.value

    def close(self):
        if getattr(self, "h", None):
            L.lib().sg_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Lines:
    offsets: torch.Tensor      # int64 [n_lines + 1]
    vertices: torch.Tensor     # float32 [n_vertices, 3] world
    status: torch.Tensor       # uint8 [n_lines]
    margin: torch.Tensor       # float32 [n_lines]
    source: torch.Tensor       # int32 [n_lines]

    def lengths(self):
        return self.offsets[1:] - self.offsets[:-1]


@dataclass
class JoinedLines:
    offsets: torch.Tensor      # int64 [n_seeds + 1]
    vertices: torch.Tensor     # float32 [n_vertices, 3] world: backward part reversed, then forward
    seed_vertex: torch.Tensor  # int64 [n_seeds]: index of the seed in its polyline (-1: OUT seed)

    def lengths(self):
        return self.offsets[1:] - self.offsets[:-1]


def _vec3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


def seeds_rake(a, b, n: int, device="cuda", stream=None) -> torch.Tensor:
    """n seeds evenly spaced on the world segment a..b (device kernel)."""
    out = torch.empty((max(int(n), 1), 3), dtype=torch.float32, device=device)
    va, vb = _vec3(a), _vec3(b)
    call("sg_seeds_rake", _ptr(va), _ptr(vb), int(n), _ptr(out), _stream(stream))
    return out[:int(n)]


def seeds_plane(origin, u, v, nu: int, nv: int, device="cuda", stream=None) -> torch.Tensor:
    """nu x nv seeds evenly spaced on the parallelogram origin + s u + t v (device kernel)."""
    n = int(nu) * int(nv)
    out = torch.empty((max(n, 1), 3), dtype=torch.float32, device=device)
    vo, vu, vv = _vec3(origin), _vec3(u), _vec3(v)
    call("sg_seeds_plane", _ptr(vo), _ptr(vu), _ptr(vv), int(nu), int(nv), _ptr(out), _stream(stream))
    return out[:n]


def seeds_box(lo, hi, n: int, seed: int, stream_id: int = 0, device="cuda", stream=None) -> torch.Tensor:
    """n seeds uniform at random in the world box [lo, hi] (SplitMix64 stream, device kernel)."""
    out = torch.empty((max(int(n), 1), 3), dtype=torch.float32, device=device)
    vl, vh = _vec3(lo), _vec3(hi)
    call("sg_seeds_box", _ptr(vl), _ptr(vh), int(n), int(seed), int(stream_id), _ptr(out), _stream(stream))
    return out[:int(n)]


def tracer_params(dt, max_steps=1000, mode="streamline", kernel="persistent", eps=1e-6, tie_cells=1e-3,
                  tie_eps_rel=1e-3, inject_steps=1, block_size=0, blocks_per_sm=0, steps_per_round=0,
                  max_rounds=0, drain_steps=0, direction="forward", brick_window=0) -> L.sg_tracer_params:
    p = L.sg_tracer_params()
    call("sg_tracer_params_default", ctypes.byref(p))
    p.mode = {"streamline": L.SG_STREAMLINE, "streakline": L.SG_STREAKLINE, "pathline": L.SG_PATHLINE}[mode]
    p.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    p.dt = float(dt)
    p.max_steps = int(max_steps)
    p.eps = float(eps)
    p.tie_cells = float(tie_cells)
    p.tie_eps_rel = float(tie_eps_rel)
    p.inject_steps = int(inject_steps)
    p.block_size = int(block_size)
    p.blocks_per_sm = int(blocks_per_sm)
    p.steps_per_round = int(steps_per_round)
    p.max_rounds = int(max_rounds)
    p.drain_steps = int(drain_steps)
    p.direction = DIRECTIONS[direction] if isinstance(direction, str) else int(direction)
    p.brick_window = int(brick_window)
    return p


class Tracer:
    """Streamline or streakline tracer (the paper's Tracer: step / trace / getLines)."""

    def __init__(self, ctx: Context, field: Field, capacity: int, **params):
        self.ctx = ctx
        self.field = field
        self.params = tracer_params(**params)
        self.capacity = int(capacity)
        nbytes = ctypes.c_size_t()
        call("sg_tracer_required_bytes", ctx.h, field.h, ctypes.byref(self.params), self.capacity,
             ctypes.byref(nbytes))
        self.nbytes = nbytes.value
        self.workspace = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=f"cuda:{ctx.device}")
        h = ctypes.c_void_p()
        call("sg_tracer_create", ctx.h, field.h, ctypes.byref(self.params), self.capacity, _ptr(self.workspace),
             self.nbytes, ctypes.byref(h))
        self.h = h
        self._seeds = None

    def upload_seeds(self, xyz, stream=None):
        """xyz: (n, 3) float32 world positions (torch tensor on any device, or numpy)."""
        if isinstance(xyz, np.ndarray):
            xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32))
        assert xyz.dtype == torch.float32
        xyz = xyz.contiguous()
        self._seeds = xyz           # keep alive until the copy is done
        call("sg_tracer_upload_seeds", self.h, _ptr(xyz), int(xyz.shape[0]), _stream(stream))

    def step(self, n_steps: int = 1, sync: bool = True, stream=None):
        act = ctypes.c_int32(0)
        call("sg_tracer_step", self.h, int(n_steps), ctypes.byref(act) if sync else None, _stream(stream))
        return bool(act.value) if sync else None

    def trace(self, stream=None):
        call("sg_tracer_trace", self.h, _stream(stream))

    def trace_timed(self, stream=None, per_round=False):
        """Host-driven rounds with CUDA events around each advection kernel:
        returns (summed kernel ms, launches[, per-round ms, per-round particles])."""
        ms = ctypes.c_double()
        n = ctypes.c_int32()
        cap = 4096
        rms = np.zeros(cap, dtype=np.float32)
        rq = np.zeros(cap, dtype=np.uint32)
        call("sg_tracer_trace_timed", self.h, ctypes.byref(ms), ctypes.byref(n), _ptr(rms), _ptr(rq), cap,
             _stream(stream))
        if per_round:
            k = min(n.value, cap)
            return ms.value, n.value, rms[:k].copy(), rq[:k].copy()
        return ms.value, n.value

    def check(self, stream=None) -> int:
        r = ctypes.c_int32()
        call("sg_tracer_check", self.h, ctypes.byref(r), _stream(stream))
        return r.value

    def sizes(self, stream=None):
        nl = ctypes.c_int64()
        nv = ctypes.c_int64()
        call("sg_tracer_get_lines", self.h, ctypes.byref(nl), ctypes.byref(nv), None, None, None, None, None,
             _stream(stream))
        return nl.value, nv.value

    def get_lines(self, device="cuda", stream=None) -> Lines:
        """CSR lines; device 'cuda' (the tracer's GPU) or 'pinned' (page-locked host)."""
        nl, nv = self.sizes(stream)
        if device == "pinned":
            kw = dict(pin_memory=True)
        else:
            kw = dict(device=f"cuda:{self.ctx.device}")
        off = torch.empty(nl + 1, dtype=torch.int64, **kw)
        vert = torch.empty((max(nv, 1), 3), dtype=torch.float32, **kw)
        st = torch.empty(max(nl, 1), dtype=torch.uint8, **kw)
        mg = torch.empty(max(nl, 1), dtype=torch.float32, **kw)
        src = torch.empty(max(nl, 1), dtype=torch.int32, **kw)
        call("sg_tracer_get_lines", self.h, None, None, _ptr(off), _ptr(vert), _ptr(st), _ptr(mg), _ptr(src),
             _stream(stream))
        return Lines(off, vert[:nv], st[:nl], mg[:nl], src[:nl])

    def get_lines_overlapped(self, out=None, stream=None) -> Lines:
        """CSR lines into page-locked host tensors, copied on the tracer's copy
        stream while work enqueued later on `stream` runs.  `out` (a Lines of
        pinned tensors large enough, e.g. from an earlier call) is reused when
        given.  The tensors are complete after wait_lines(stream) and a
        synchronisation of `stream`."""
        nl = ctypes.c_int64()
        nv = ctypes.c_int64()
        call("sg_tracer_get_lines_overlapped", self.h, ctypes.byref(nl), ctypes.byref(nv), None, None, None, None,
             _stream(stream))
        nl, nv = nl.value, nv.value
        if (out is None or out.offsets.numel() < nl + 1 or out.vertices.shape[0] < nv
                or out.status.numel() < nl or out.margin.numel() < nl):
            off = torch.empty(nl + 1, dtype=torch.int64, pin_memory=True)
            vert = torch.empty((max(nv, 1), 3), dtype=torch.float32, pin_memory=True)
            st = torch.empty(max(nl, 1), dtype=torch.uint8, pin_memory=True)
            mg = torch.empty(max(nl, 1), dtype=torch.float32, pin_memory=True)
        else:
            off, vert, st, mg = out.offsets, out.vertices, out.status, out.margin
        call("sg_tracer_get_lines_overlapped", self.h, None, None, _ptr(off), _ptr(vert), _ptr(st), _ptr(mg),
             _stream(stream))
        return Lines(off[:nl + 1], vert[:nv], st[:nl], mg[:nl], None)

    def wait_lines(self, stream=None):
        """Makes `stream` wait for the host copies of the last overlapped readout."""
        call("sg_tracer_wait_lines", self.h, _stream(stream))

    def get_joined(self, stream=None) -> JoinedLines:
        """Bidirectional tracers: one polyline per seed through the seed (device)."""
        nl = ctypes.c_int64()
        nv = ctypes.c_int64()
        call("sg_tracer_get_joined", self.h, ctypes.byref(nl), ctypes.byref(nv), None, None, None, _stream(stream))
        dev = f"cuda:{self.ctx.device}"
        off = torch.empty(nl.value + 1, dtype=torch.int64, device=dev)
        vert = torch.empty((max(nv.value, 1), 3), dtype=torch.float32, device=dev)
        sv = torch.empty(max(nl.value, 1), dtype=torch.int64, device=dev)
        call("sg_tracer_get_joined", self.h, None, None, _ptr(off), _ptr(vert), _ptr(sv), _stream(stream))
        return JoinedLines(off, vert[:nv.value], sv[:nl.value])

    def total_steps(self, stream=None) -> int:
        n = ctypes.c_int64()
        call("sg_tracer_total_steps", self.h, ctypes.byref(n), _stream(stream))
        return n.value

    # -- partition over data (see pod.py for the exchange between ranks)

    def pod_setup(self, brick_owner, rank: int, world: int):
        owner = np.ascontiguousarray(np.asarray(brick_owner, dtype=np.int32))
        call("sg_tracer_pod_setup", self.h, _ptr(owner), int(rank), int(world))
        self.pod_world = int(world)

    def pod_begin(self, stream=None) -> int:
        n = ctypes.c_int64()
        call("sg_tracer_pod_begin", self.h, ctypes.byref(n), _stream(stream))
        return n.value

    def pod_round(self, stream=None):
        """One round; returns (local queue length, export counts per rank)."""
        n = ctypes.c_int64()
        ex = np.zeros(self.pod_world, dtype=np.int64)
        call("sg_tracer_pod_round", self.h, ctypes.byref(n), _ptr(ex), _stream(stream))
        return n.value, ex

    def pod_export(self, dest: int, count: int, stream=None) -> torch.Tensor:
        """The export segment for rank dest as a uint8 tensor of count x 32 bytes (device)."""
        out = torch.empty(max(int(count), 1) * 32, dtype=torch.uint8, device=f"cuda:{self.ctx.device}")
        call("sg_tracer_pod_export", self.h, int(dest), _ptr(out), _stream(stream))
        return out[:int(count) * 32]

    def pod_import(self, records: torch.Tensor, stream=None):
        records = records.contiguous()
        assert records.dtype == torch.uint8 and records.numel() % 32 == 0
        self._imported = records                 # alive until the copy is done
        call("sg_tracer_pod_import", self.h, _ptr(records), records.numel() // 32, _stream(stream))

    def pod_queued(self) -> int:
        n = ctypes.c_int64()
        call("sg_tracer_pod_queued", self.h, ctypes.byref(n))
        return n.value

    def line_buffers(self):
        """Views (torch, device) of the tracer's line buffers: slab [n_lines, W, 3],
        length [n_lines] int32 (uint32 bits), status [n_lines] uint8, margin [n_lines]."""
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        nl = ctypes.c_int64()
        w = ctypes.c_int64()
        call("sg_tracer_line_buffers", self.h, *[ctypes.byref(x) for x in ptrs], ctypes.byref(nl), ctypes.byref(w))
        base = self.workspace.data_ptr()

        def view(ptr, nbytes, dtype, shape):
            off = ptr.value - base
            assert 0 <= off and off + nbytes <= self.workspace.numel()
            return self.workspace[off:off + nbytes].view(dtype).view(shape)

        n, W = nl.value, w.value
        slab = view(ptrs[0], n * W * 12, torch.float32, (n, W, 3))
        length = view(ptrs[1], n * 4, torch.int32, (n,))
        status = view(ptrs[2], n, torch.uint8, (n,))
        margin = view(ptrs[3], n * 4, torch.float32, (n,))
        return slab, length, status, margin

    def close(self):
        if getattr(self, "h", None):
            L.lib().sg_tracer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UMesh:
    """Unstructured field (tetrahedra, pyramids, prisms, hexahedra) with the
    velocity at its vertices; a hierarchy for point location (sg_umesh_*)."""

    def __init__(self, ctx: Context, mesh: dict, tau: float = 0.0):
        self.ctx = ctx
        X = np.ascontiguousarray(mesh["vertices"], dtype=np.float32)
        V = np.ascontiguousarray(mesh["velocity"], dtype=np.float32)
        idx = np.ascontiguousarray(mesh["cell_vertices"], dtype=np.int32)
        off = np.ascontiguousarray(mesh["cell_offsets"], dtype=np.int64)
        typ = np.ascontiguousarray(mesh["cell_types"], dtype=np.uint8)
        self.n_cells = len(typ)
        nbytes = ctypes.c_size_t()
        call("sg_umesh_required_bytes", self.n_cells, ctypes.byref(nbytes))
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=f"cuda:{ctx.device}")
        h = ctypes.c_void_p()
        call("sg_umesh_create", ctx.h, _ptr(X), _ptr(V), len(X), _ptr(idx), _ptr(off), _ptr(typ), self.n_cells,
             float(tau), _ptr(self.workspace), nbytes.value, ctypes.byref(h))
        self.h = h

    def sample(self, points, stream=None):
        """(velocity [n, 3] float32, cell [n] int64) at world points (device)."""
        pts = torch.as_tensor(points, dtype=torch.float32).to(f"cuda:{self.ctx.device}").contiguous()
        n = pts.shape[0]
        v = torch.empty((max(n, 1), 3), dtype=torch.float32, device=pts.device)
        c = torch.empty(max(n, 1), dtype=torch.int64, device=pts.device)
        call("sg_umesh_sample", self.h, _ptr(pts), n, _ptr(v), _ptr(c), _stream(stream))
        return v[:n], c[:n]

    def trace(self, seeds, dt: float, max_steps: int, eps: float = 1e-6, stream=None) -> Lines:
        """Streamlines from world seeds, compacted to CSR (device).  Every
        buffer is allocated, and every call enqueued, on `stream` (the current
        stream if None), which the call synchronises once to size the CSR."""
        dev = f"cuda:{self.ctx.device}"
        strm = torch.cuda.current_stream(dev) if stream is None else stream
        with torch.cuda.stream(strm):
            s = torch.as_tensor(seeds, dtype=torch.float32).to(dev).contiguous()
            n = s.shape[0]
            W = int(max_steps) + 1
            slab = torch.empty((max(n, 1), W, 3), dtype=torch.float32, device=dev)
            length = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            st = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
            mg = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
            call("sg_umesh_trace", self.h, _ptr(s), n, float(dt), int(max_steps), float(eps), _ptr(slab),
                 _ptr(length), _ptr(st), _ptr(mg), _stream(strm))
            nsc = ctypes.c_size_t()
            call("sg_lines_compact_scratch_bytes", n, ctypes.byref(nsc))
            scratch = torch.empty(max(nsc.value, 8), dtype=torch.uint8, device=dev)
            off = torch.empty(n + 1, dtype=torch.int64, device=dev)
            call("sg_lines_compact", _ptr(slab), W, _ptr(length), n, _ptr(scratch), nsc.value, _ptr(off), None,
                 _stream(strm))
            total = int(off[n].item()) if n else 0
            vert = torch.empty((max(total, 1), 3), dtype=torch.float32, device=dev)
            call("sg_lines_compact", _ptr(slab), W, _ptr(length), n, _ptr(scratch), nsc.value, _ptr(off),
                 _ptr(vert), _stream(strm))
            src = torch.arange(n, dtype=torch.int32, device=dev)
        return Lines(off, vert[:total], st[:n], mg[:n], src)

    def close(self):
        if getattr(self, "h", None):
            L.lib().sg_umesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Continuous batching of streamline requests (sg_batch_*): requests join
    between runs and leave when their last line stops."""

    def __init__(self, ctx: Context, max_lines: int, slab_bytes: int, layout="cell8", max_requests=1024,
                 max_fields=16, max_bricks=4096, block_size=0, blocks_per_sm=0, steps_per_round=0, drain_steps=0):
        self.ctx = ctx
        d = L.sg_batch_desc()
        d.max_lines = int(max_lines)
        d.slab_bytes = int(slab_bytes)
        d.max_requests = int(max_requests)
        d.max_fields = int(max_fields)
        d.max_bricks = int(max_bricks)
        d.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        d.block_size = int(block_size)
        d.blocks_per_sm = int(blocks_per_sm)
        d.steps_per_round = int(steps_per_round)
        d.drain_steps = int(drain_steps)
        self.desc = d
        nbytes = ctypes.c_size_t()
        call("sg_batch_required_bytes", ctx.h, ctypes.byref(d), ctypes.byref(nbytes))
        self.nbytes = nbytes.value
        self.workspace = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=f"cuda:{ctx.device}")
        h = ctypes.c_void_p()
        call("sg_batch_create", ctx.h, ctypes.byref(d), _ptr(self.workspace), self.nbytes, ctypes.byref(h))
        self.h = h
        self._keep = {}

    def capacity(self):
        fl = ctypes.c_int64()
        sb = ctypes.c_int64()
        fr = ctypes.c_int32()
        call("sg_batch_capacity", self.h, ctypes.byref(fl), ctypes.byref(sb), ctypes.byref(fr))
        return fl.value, sb.value, fr.value

    def submit(self, field: Field, xyz, dt, max_steps, eps=1e-6, tie_cells=1e-3, tie_eps_rel=1e-3, stream=None):
        """Returns the request id, or None when the request does not fit now."""
        if isinstance(xyz, np.ndarray):
            xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32))
        xyz = xyz.contiguous()
        p = tracer_params(dt=dt, max_steps=max_steps, eps=eps, tie_cells=tie_cells, tie_eps_rel=tie_eps_rel)
        rid = ctypes.c_int64()
        code = L.lib().sg_batch_submit(self.h, field.h, _ptr(xyz), int(xyz.shape[0]), ctypes.byref(p),
                                       ctypes.byref(rid), _stream(stream))
        if code == L.SG_ERR_OOM:
            return None
        L.check("sg_batch_submit", code)
        self._keep[rid.value] = xyz
        return rid.value

    def run(self, max_rounds: int = 0, stream=None):
        call("sg_batch_run", self.h, int(max_rounds), _stream(stream))

    def finished(self, stream=None):
        cap = 4096
        ids = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int32()
        call("sg_batch_finished", self.h, _ptr(ids), cap, ctypes.byref(n), _stream(stream))
        return [int(x) for x in ids[: n.value]]

    def get_lines(self, rid: int, device="cuda", stream=None) -> Lines:
        nl = ctypes.c_int64()
        nv = ctypes.c_int64()
        call("sg_batch_get_lines", self.h, rid, ctypes.byref(nl), ctypes.byref(nv), None, None, None, None,
             _stream(stream))
        kw = dict(pin_memory=True) if device == "pinned" else dict(device=f"cuda:{self.ctx.device}")
        off = torch.empty(nl.value + 1, dtype=torch.int64, **kw)
        vert = torch.empty((max(nv.value, 1), 3), dtype=torch.float32, **kw)
        st = torch.empty(max(nl.value, 1), dtype=torch.uint8, **kw)
        mg = torch.empty(max(nl.value, 1), dtype=torch.float32, **kw)
        call("sg_batch_get_lines", self.h, rid, None, None, _ptr(off), _ptr(vert), _ptr(st), _ptr(mg),
             _stream(stream))
        src = torch.zeros(max(nl.value, 1), dtype=torch.int32)
        return Lines(off, vert[: nv.value], st[: nl.value], mg[: nl.value], src[: nl.value])

    def release(self, rid: int, stream=None):
        call("sg_batch_release", self.h, rid, _stream(stream))
        self._keep.pop(rid, None)

    def close(self):
        if getattr(self, "h", None):
            L.lib().sg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
