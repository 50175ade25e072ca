"""The C ABI library builds, loads and exports what include/tigre103.h
declares; argument validation runs before any CUDA call (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tigre103.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1905_03748_gb300.csrc import build
    return ctypes.CDLL(build.build())


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"TIGRE_API\s+[\w\s\*]+?\b(tigre_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["tigre_geometry_create", "tigre_geometry_destroy", "tigre_forward",
              "tigre_backward", "tigre_tv_step", "tigre_sirt", "tigre_sart", "tigre_cgls",
              "tigre_last_error"]:
        assert n in names


def test_binding_flag_values_match_header():
    from paper_1905_03748_gb300 import tigre
    text = open(HEADER).read()
    flags = dict(re.findall(r"#define\s+(TIGRE_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+)u", text))
    assert {"TIGRE_HOST_RESIDENT", "TIGRE_GRAPH", "TIGRE_OUT_OF_CORE", "TIGRE_X0_ZERO"} <= set(flags)
    for name, value in flags.items():
        assert getattr(tigre, name) == int(value, 16), name


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1905_03748_gb300 import tigre
    for name in declared_functions():
        assert name in tigre.EXPORTED and callable(getattr(tigre, name)), name


def test_invalid_geometry_rejected_before_cuda(lib):
    from paper_1905_03748_gb300 import tigre
    lib.tigre_geometry_create.restype = ctypes.c_int
    lib.tigre_last_error.restype = ctypes.c_char_p
    ang = np.zeros(3)
    h = ctypes.c_void_p()
    good = dict(DSO=100.0, DSD=150.0, n_voxel=(8, 8, 8), d_voxel=(1.0, 1.0, 1.0),
                off_origin=(0.0, 0.0, 0.0), n_det=(8, 8), d_det=(1.0, 1.0), off_det=(0.0, 0.0),
                accuracy=0.5)
    bad = [dict(good, DSD=90.0), dict(good, n_voxel=(0, 8, 8)), dict(good, d_det=(1.0, -1.0)),
           dict(good, DSO=5.0), dict(good, accuracy=float("nan"))]
    for b in bad:
        d = tigre.make_desc(b)
        st = lib.tigre_geometry_create(ctypes.byref(d), ang.ctypes.data_as(ctypes.c_void_p), 3,
                                       ctypes.byref(h))
        assert st == tigre.TIGRE_ERR_INVALID_ARG, b
        assert h.value is None
        assert lib.tigre_last_error()
    d = tigre.make_desc(good)
    st = lib.tigre_geometry_create(ctypes.byref(d), ang.ctypes.data_as(ctypes.c_void_p), 0,
                                   ctypes.byref(h))
    assert st == tigre.TIGRE_ERR_INVALID_ARG


def test_solver_defaults(lib):
    from paper_1905_03748_gb300 import tigre
    o = tigre.tigre_solver_opts_default()
    assert o.n_iter == 10 and o.lambda_ == 1.0 and o.subset_size == 20
    assert o.bp_weight == tigre.TIGRE_BP_MATCHED and o.storage == tigre.TIGRE_F32


def test_allocator_needs_both_functions_and_resets():
    from paper_1905_03748_gb300 import tigre
    alloc = tigre.ALLOC_FN(lambda n, s, c: 0)
    assert tigre._lib.tigre_set_allocator(alloc, tigre.FREE_FN(), None) == tigre.TIGRE_ERR_INVALID_ARG
    tigre.tigre_set_allocator(lambda n, s: 0, lambda p, s: None)
    tigre.tigre_set_allocator(None, None)
