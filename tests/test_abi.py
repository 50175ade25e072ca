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


C_PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "tigre103.h"

int main(void)
{
    tigre_solver_opts o;
    if (tigre_solver_opts_default(&o) != TIGRE_OK) return 1;
    tigre_geometry_desc d = {0};
    d.DSO = 1000.0;
    d.DSD = 1536.0;
    for (int k = 0; k < 3; ++k) {
        d.n_voxel[k] = 512;
        d.d_voxel[k] = 0.5;
    }
    d.n_det[0] = d.n_det[1] = 512;
    d.d_det[0] = d.d_det[1] = 0.8807;
    d.accuracy = 0.5;
    static double ang[360];
    for (int a = 0; a < 360; ++a) ang[a] = 2.0 * 3.14159265358979323846 * a / 360.0;
    int placement = 0, pairs = 0;
    int64_t slab = 0, groups = 0;
    double drift = 0.0;
    if (tigre_cgls_ooc_plan_desc(&d, ang, 360, (int64_t)4e10, &placement, &slab) != TIGRE_OK)
        return 2;
    if (tigre_forward_angle_groups(&d, ang, 360, 2, NULL, 0, &groups, &drift, &pairs) != TIGRE_OK)
        return 3;
    const tigre_status bad = tigre_cgls_ooc_plan_desc(&d, ang, 360, 0, &placement, &slab);
    printf("%d %g %d %d %lld %lld %.6f %d %d %s\n", o.n_iter, o.lambda, o.subset_size,
           placement, (long long)slab, (long long)groups, drift, pairs, (int)bad,
           tigre_last_error()[0] ? "msg" : "nomsg");
    return 0;
}
"""


def test_plain_c_program_uses_the_abi(tmp_path):
    """The header is C99 (gcc -pedantic, no warnings) and a C program linked
    against the library gets the same host-side answers as the binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1905_03748_gb300 import synth, tigre
    from paper_1905_03748_gb300.csrc import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), lib,
                         "-Wl,-rpath," + os.path.dirname(lib), "-lm"],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stderr)
    f = run.stdout.split()
    geo, ang = synth.workload("cgls_512")
    opts = tigre.tigre_solver_opts_default()
    assert (int(f[0]), float(f[1]), int(f[2])) == (opts.n_iter, opts.lambda_, opts.subset_size)
    assert (int(f[3]), int(f[4])) == tigre.tigre_cgls_ooc_plan_desc(geo, ang, int(4e10))
    tab, drift, pairs = tigre.tigre_forward_angle_groups(geo, ang, 2)
    assert int(f[5]) == len(tab) and float(f[6]) == pytest.approx(drift, rel=1e-3)
    assert bool(int(f[7])) == pairs
    assert int(f[8]) == tigre.TIGRE_ERR_INVALID_ARG and f[9] == "msg"

