"""ctypes binding of libstreamgb (include/streamgb.h): argument marshalling only.

Every function of the C ABI is available under its own name on ``lib()``;
the structures mirror ``sg_field_desc`` and ``sg_tracer_params``.  Loading
fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstreamgb.so")

# status codes
SG_OK = 0
SG_ERR_INVALID_ARG = -1
SG_ERR_OOM = -2
SG_ERR_CUDA = -3
SG_ERR_ROUND_LIMIT = -4
SG_ERR_TIMEOUT = -5
SG_ERR_STATE = -6
SG_ERR_UNSUPPORTED = -7
ERR_NAMES = {0: "SG_OK", -1: "SG_ERR_INVALID_ARG", -2: "SG_ERR_OOM", -3: "SG_ERR_CUDA",
             -4: "SG_ERR_ROUND_LIMIT", -5: "SG_ERR_TIMEOUT", -6: "SG_ERR_STATE", -7: "SG_ERR_UNSUPPORTED"}

SG_F32, SG_BF16, SG_F16, SG_FX21 = 0, 1, 2, 3
SG_LAYOUT_LINEAR, SG_LAYOUT_TILED4, SG_LAYOUT_CELL8, SG_FIELD_GLOBAL = 0, 1, 2, 16
SG_STREAMLINE, SG_STREAKLINE = 0, 1
SG_KERNEL_PERSISTENT, SG_KERNEL_PER_SEED, SG_KERNEL_PER_STEP, SG_KERNEL_LOCKSTEP = 0, 1, 2, 3
SG_DIR_FORWARD, SG_DIR_BACKWARD, SG_DIR_BOTH = 0, 1, 2
SG_PATHLINE = 2
SG_LINE_ACTIVE, SG_LINE_MAXSTEPS, SG_LINE_EXIT, SG_LINE_STAGNANT = 0, 1, 2, 3
SG_LINE_NANFIELD, SG_LINE_OUT, SG_LINE_HALO, SG_LINE_TIE = 4, 5, 6, 0x80


class sg_field_desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
                ("bricks", ctypes.c_int32 * 3), ("ghost", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("n_slots", ctypes.c_int32), ("slice_dt", ctypes.c_double)]


class sg_tracer_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("kernel", ctypes.c_int32), ("dt", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("eps", ctypes.c_float), ("tie_cells", ctypes.c_float),
                ("tie_eps_rel", ctypes.c_float), ("inject_steps", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("steps_per_round", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("drain_steps", ctypes.c_int32), ("direction", ctypes.c_int32),
                ("brick_window", ctypes.c_int32)]


class sg_batch_desc(ctypes.Structure):
    _fields_ = [("max_lines", ctypes.c_int64), ("slab_bytes", ctypes.c_int64), ("max_requests", ctypes.c_int32),
                ("max_fields", ctypes.c_int32), ("max_bricks", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("steps_per_round", ctypes.c_int32), ("drain_steps", ctypes.c_int32)]


class StreamGBError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} -> {ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


P = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
sz = ctypes.c_size_t
PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (argtypes, restype)
SIGNATURES = {
    "sg_last_error": ([ctypes.c_char_p, sz], sz),
    "sg_version": ([], i32),
    "sg_context_create": ([i32, PP], i32),
    "sg_context_destroy": ([P], i32),
    "sg_context_sm_count": ([P, ctypes.POINTER(i32)], i32),
    "sg_field_required_bytes": ([ctypes.POINTER(sg_field_desc), ctypes.POINTER(sz)], i32),
    "sg_field_create": ([P, ctypes.POINTER(sg_field_desc), P, sz, PP], i32),
    "sg_field_destroy": ([P], i32),
    "sg_field_brick_cells": ([P, ctypes.POINTER(i64)], i32),
    "sg_field_set_global": ([P, i32, P, P], i32),
    "sg_field_set_brick": ([P, i32, i32, i32, i32, P, P], i32),
    "sg_field_stream_slice": ([P, i32, P, P], i32),
    "sg_field_max_speed": ([P, i32, ctypes.POINTER(ctypes.c_double), P], i32),
    "sg_field_read_brick": ([P, i32, i32, i32, i32, P, ctypes.POINTER(ctypes.c_float), P], i32),
    "sg_tracer_params_default": ([ctypes.POINTER(sg_tracer_params)], i32),
    "sg_tracer_required_bytes": ([P, P, ctypes.POINTER(sg_tracer_params), i64, ctypes.POINTER(sz)], i32),
    "sg_tracer_create": ([P, P, ctypes.POINTER(sg_tracer_params), i64, P, sz, PP], i32),
    "sg_tracer_destroy": ([P], i32),
    "sg_tracer_upload_seeds": ([P, P, i64, P], i32),
    "sg_tracer_step": ([P, i32, ctypes.POINTER(i32), P], i32),
    "sg_tracer_trace": ([P, P], i32),
    "sg_tracer_check": ([P, ctypes.POINTER(i32), P], i32),
    "sg_tracer_trace_timed": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), P, P, i32, P], i32),
    "sg_tracer_get_lines": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64), P, P, P, P, P, P], i32),
    "sg_tracer_total_steps": ([P, ctypes.POINTER(i64), P], i32),
    "sg_tracer_get_lines_overlapped": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64), P, P, P, P, P], i32),
    "sg_tracer_wait_lines": ([P, P], i32),
    "sg_tracer_get_joined": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64), P, P, P, P], i32),
    "sg_seeds_rake": ([P, P, i64, P, P], i32),
    "sg_umesh_required_bytes": ([i64, ctypes.POINTER(ctypes.c_size_t)], i32),
    "sg_umesh_create": ([P, P, P, i64, P, P, P, i64, ctypes.c_float, P, ctypes.c_size_t, ctypes.POINTER(P)], i32),
    "sg_umesh_destroy": ([P], i32),
    "sg_umesh_sample": ([P, P, i64, P, P, P], i32),
    "sg_umesh_trace": ([P, P, i64, ctypes.c_double, i32, ctypes.c_float, P, P, P, P, P], i32),
    "sg_tracer_pod_setup": ([P, P, i32, i32], i32),
    "sg_tracer_pod_begin": ([P, ctypes.POINTER(i64), P], i32),
    "sg_tracer_pod_round": ([P, ctypes.POINTER(i64), P, P], i32),
    "sg_tracer_pod_export": ([P, i32, P, P], i32),
    "sg_tracer_pod_import": ([P, P, i64, P], i32),
    "sg_tracer_pod_queued": ([P, ctypes.POINTER(i64)], i32),
    "sg_tracer_line_buffers": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
    "sg_seeds_plane": ([P, P, P, i64, i64, P, P], i32),
    "sg_seeds_box": ([P, P, i64, ctypes.c_uint64, ctypes.c_uint64, P, P], i32),
    "sg_lines_compact_static": ([P, i64, P, i64, P, P, P], i32),
    "sg_lines_compact_scratch_bytes": ([i64, ctypes.POINTER(sz)], i32),
    "sg_lines_compact": ([P, i64, P, i64, P, sz, P, P, P], i32),
    "sg_batch_required_bytes": ([P, ctypes.POINTER(sg_batch_desc), ctypes.POINTER(sz)], i32),
    "sg_batch_create": ([P, ctypes.POINTER(sg_batch_desc), P, sz, PP], i32),
    "sg_batch_destroy": ([P], i32),
    "sg_batch_capacity": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)], i32),
    "sg_batch_submit": ([P, P, P, i64, ctypes.POINTER(sg_tracer_params), ctypes.POINTER(i64), P], i32),
    "sg_batch_run": ([P, i32, P], i32),
    "sg_batch_finished": ([P, P, i32, ctypes.POINTER(i32), P], i32),
    "sg_batch_get_lines": ([P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), P, P, P, P, P], i32),
    "sg_batch_release": ([P, i64, P], i32),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libstreamgb.so is not built ({LIB_PATH}); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().sg_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(fn_name: str, code: int) -> int:
    if code != SG_OK:
        raise StreamGBError(fn_name, code, last_error())
    return code


def call(fn_name: str, *args) -> int:
    """Calls a C ABI function and raises StreamGBError on a non-zero status."""
    return check(fn_name, getattr(lib(), fn_name)(*args))
