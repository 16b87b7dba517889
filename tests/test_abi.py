"""CPU checks of the C ABI: the library builds, loads and exports every
function that include/streamgb.h declares; host-side argument checks and size
queries work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:sg_status|size_t|int32_t)\s+(sg_\w+)\s*\(", text, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_02627_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) <= set(lib.SIGNATURES), set(names) - set(lib.SIGNATURES)


def test_version_and_defaults(lib):
    L = lib.lib()
    assert L.sg_version() >= 100
    p = lib.sg_tracer_params()
    assert L.sg_tracer_params_default(ctypes.byref(p)) == 0
    assert p.max_steps == 1000 and abs(p.eps - 1e-6) < 1e-12 and p.mode == 0
    assert L.sg_tracer_params_default(None) == lib.SG_ERR_INVALID_ARG
    assert "NULL" in lib.last_error()


def test_field_size_query_and_validation(lib):
    from paper_2606_02627_gb300 import api
    L = lib.lib()
    d = api.field_desc((512, 512, 512), (0, 0, 0), (0.0123, 0.0123, 0.0123), bricks=(4, 4, 4))
    n = ctypes.c_size_t()
    assert L.sg_field_required_bytes(ctypes.byref(d), ctypes.byref(n)) == 0
    # 64 bricks of 131^3 samples, 16 bytes each, plus scales and scratch
    assert 64 * 131 ** 3 * 16 <= n.value < 64 * 131 ** 3 * 16 + 2 ** 20
    d16 = api.field_desc((512, 512, 512), (0, 0, 0), (0.0123,) * 3, bricks=(4, 4, 4), dtype="bf16")
    n16 = ctypes.c_size_t()
    assert L.sg_field_required_bytes(ctypes.byref(d16), ctypes.byref(n16)) == 0
    assert n16.value < 0.51 * n.value
    bad = api.field_desc((4, 4, 4), (0, 0, 0), (1, 1, 1), bricks=(4, 1, 1))
    assert L.sg_field_required_bytes(ctypes.byref(bad), ctypes.byref(n)) == lib.SG_ERR_INVALID_ARG
    assert "last brick" in lib.last_error()
    neg = api.field_desc((8, 8, 8), (0, 0, 0), (1, -1, 1))
    assert L.sg_field_required_bytes(ctypes.byref(neg), ctypes.byref(n)) == lib.SG_ERR_INVALID_ARG
    glob = api.field_desc((8, 8, 8), (0, 0, 0), (1, 1, 1), bricks=(2, 1, 1), layout="global")
    assert L.sg_field_required_bytes(ctypes.byref(glob), ctypes.byref(n)) == lib.SG_ERR_INVALID_ARG


def test_umesh_size_query(lib):
    """A mesh's workspace: 256-B cell records, at most one 32-B hierarchy node
    per cell (leaves of 2 to 4 cells), a 4-B index per cell, each part
    256-byte aligned."""
    L = lib.lib()
    up = lambda x: (x + 255) // 256 * 256
    n = ctypes.c_size_t()
    for cells in (0, 1, 2, 5, 1000, 2_097_152):
        assert L.sg_umesh_required_bytes(cells, ctypes.byref(n)) == 0
        assert n.value == up(256 * cells) + up(32 * max(cells, 1)) + up(4 * cells), cells
    assert L.sg_umesh_required_bytes(-1, ctypes.byref(n)) == lib.SG_ERR_INVALID_ARG


def test_context_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = lib.lib()
    h = ctypes.c_void_p()
    rc = L.sg_context_create(0, ctypes.byref(h))
    assert rc in (lib.SG_ERR_CUDA, lib.SG_ERR_INVALID_ARG)
    assert lib.last_error()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_02627_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "liboracle" not in text, fn
