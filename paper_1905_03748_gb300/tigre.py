"""Thin ctypes binding of libtigre103 (the C ABI in include/tigre103.h).

Every function keeps the C name and only marshals arguments: torch tensors
become device pointers plus a dtype code, streams become cudaStream_t
handles, and a non-OK status raises TigreError with tigre_last_error().
All computation happens in the CUDA library; there is no fallback path, and
importing this module raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtigre103.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_1905_03748_gb300.csrc.build` (no CPU fallback exists)")

_lib = ctypes.CDLL(LIB_PATH)

TIGRE_OK, TIGRE_ERR_INVALID_ARG, TIGRE_ERR_OOM, TIGRE_ERR_CUDA, TIGRE_ERR_TIMEOUT, \
    TIGRE_ERR_UNSUPPORTED = range(6)
TIGRE_F32, TIGRE_BF16, TIGRE_F16 = 0, 1, 2
TIGRE_BP_MATCHED, TIGRE_BP_FDK, TIGRE_BP_EXACT_ADJOINT = 0, 1, 2
TIGRE_HOST_RESIDENT = 0x1
TIGRE_GRAPH = 0x2

EXPORTED = ["tigre_geometry_create", "tigre_geometry_destroy", "tigre_forward", "tigre_backward",
            "tigre_tv_step", "tigre_tv_step_noalloc", "tigre_solver_opts_default", "tigre_sirt",
            "tigre_sart",
            "tigre_cgls", "tigre_cgls_begin", "tigre_cgls_iterate", "tigre_cgls_history",
            "tigre_cgls_end", "tigre_cgls_batch_begin", "tigre_cgls_batch_iterate",
            "tigre_cgls_batch_history", "tigre_cgls_batch_end", "tigre_cgls_save",
            "tigre_cgls_resume", "tigre_forward_samples", "tigre_forward_ooc", "tigre_backward_ooc",
            "tigre_cgls_ooc_plan", "tigre_geometry_set_forward_path", "tigre_forward_angle_groups",
            "tigre_cgls_ooc_plan_desc",
            "tigre_geometry_set_projector", "tigre_fdk", "tigre_rof_denoise",
            "tigre_geometry_set_brick", "tigre_tv_step_ooc", "tigre_set_allocator",
            "tigre_geometry_error_flags", "tigre_profile_enable",
            "tigre_profile_read", "tigre_launch_count", "tigre_last_error"]

_DTYPES = {torch.float32: TIGRE_F32, torch.bfloat16: TIGRE_BF16, torch.float16: TIGRE_F16}
_BP = {"matched": TIGRE_BP_MATCHED, "fdk": TIGRE_BP_FDK, "adjoint": TIGRE_BP_EXACT_ADJOINT}


class tigre_geometry_desc(ctypes.Structure):
    _fields_ = [("DSO", ctypes.c_double), ("DSD", ctypes.c_double),
                ("n_voxel", ctypes.c_int64 * 3), ("d_voxel", ctypes.c_double * 3),
                ("off_origin", ctypes.c_double * 3), ("n_det", ctypes.c_int64 * 2),
                ("d_det", ctypes.c_double * 2), ("off_det", ctypes.c_double * 2),
                ("accuracy", ctypes.c_double)]


class tigre_solver_opts(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("lambda_", ctypes.c_double),
                ("subset_size", ctypes.c_int), ("tv_steps", ctypes.c_int),
                ("tv_alpha", ctypes.c_double), ("tv_eps", ctypes.c_double),
                ("bp_weight", ctypes.c_int), ("nonneg", ctypes.c_int), ("storage", ctypes.c_int),
                ("device_budget_bytes", ctypes.c_int64), ("timeout_ms", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("cuda_stream", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_ST = ctypes.c_int
_sigs = {
    "tigre_geometry_create": [ctypes.POINTER(tigre_geometry_desc), _P, _I64, ctypes.POINTER(_P)],
    "tigre_geometry_destroy": [_P],
    "tigre_forward": [_P, _P, ctypes.c_int, _P, ctypes.c_int, _I64, _I64, _P],
    "tigre_backward": [_P, _P, ctypes.c_int, _P, ctypes.c_int, _I64, _I64, ctypes.c_int, _P],
    "tigre_tv_step": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P],
    "tigre_tv_step_noalloc": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, _P],
    "tigre_solver_opts_default": [ctypes.POINTER(tigre_solver_opts)],
    "tigre_sirt": [_P, _P, _P, ctypes.POINTER(tigre_solver_opts), _P],
    "tigre_sart": [_P, _P, _P, ctypes.POINTER(tigre_solver_opts), _P],
    "tigre_cgls": [_P, _P, _P, ctypes.POINTER(tigre_solver_opts), _P],
    "tigre_cgls_begin": [_P, _P, _P, ctypes.POINTER(tigre_solver_opts), ctypes.POINTER(_P)],
    "tigre_cgls_iterate": [_P, ctypes.c_int],
    "tigre_cgls_history": [_P, _P, ctypes.c_int],
    "tigre_cgls_end": [_P],
    "tigre_cgls_batch_begin": [_P, ctypes.c_int, _P, _P, ctypes.POINTER(tigre_solver_opts),
                               ctypes.POINTER(_P)],
    "tigre_cgls_batch_iterate": [_P, ctypes.c_int],
    "tigre_cgls_batch_history": [_P, ctypes.c_int, _P, ctypes.c_int],
    "tigre_cgls_batch_end": [_P],
    "tigre_cgls_save": [_P, _P, ctypes.c_size_t, _P, ctypes.c_size_t,
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)],
    "tigre_cgls_resume": [_P, _P, _P, _P, ctypes.c_size_t, _P, ctypes.c_size_t, ctypes.c_double,
                          ctypes.POINTER(tigre_solver_opts), ctypes.POINTER(_P)],
    "tigre_forward_samples": [_P, _I64, _I64, ctypes.POINTER(_I64)],
    "tigre_forward_ooc": [_P, _P, _P, _I64, _I64, _I64, _P],
    "tigre_backward_ooc": [_P, _P, ctypes.c_int, _P, _I64, _I64, ctypes.c_int, _I64, _I64, _P],
    "tigre_cgls_ooc_plan": [_P, _I64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64)],
    "tigre_cgls_ooc_plan_desc": [ctypes.POINTER(tigre_geometry_desc), _P, _I64, _I64,
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64)],
    "tigre_forward_angle_groups": [ctypes.POINTER(tigre_geometry_desc), _P, _I64, ctypes.c_int, _P,
                                   _I64, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int)],
    "tigre_geometry_set_forward_path": [_P, ctypes.c_int],
    "tigre_geometry_set_projector": [_P, ctypes.c_int],
    "tigre_geometry_set_brick": [_P, _I64],
    "tigre_tv_step_ooc": [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _I64, _I64, _P],
    "tigre_fdk": [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P],
    "tigre_rof_denoise": [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P],
    "tigre_geometry_error_flags": [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int],
    "tigre_profile_enable": [ctypes.c_int],
    "tigre_profile_read": [ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)],
}
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_sigs["tigre_set_allocator"] = [ALLOC_FN, FREE_FN, _P]
for _name, _args in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _ST
_lib.tigre_last_error.argtypes = []
_lib.tigre_last_error.restype = ctypes.c_char_p
_lib.tigre_launch_count.argtypes = []
_lib.tigre_launch_count.restype = ctypes.c_int64

PROF_FORWARD, PROF_BACKPROJECT, PROF_ADJOINT, PROF_TV = 0, 1, 2, 3


class TigreError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tigre status {status}: {msg}")
        self.status = status


def tigre_last_error() -> str:
    return _lib.tigre_last_error().decode()


def _check(status: int):
    if status != TIGRE_OK:
        raise TigreError(status, tigre_last_error())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in _DTYPES:
        raise TypeError(f"{name}: unsupported dtype {t.dtype}")
    return ctypes.c_void_p(t.data_ptr()), _DTYPES[t.dtype]


def make_desc(geo: dict) -> tigre_geometry_desc:
    d = tigre_geometry_desc()
    d.DSO, d.DSD = geo["DSO"], geo["DSD"]
    for i in range(3):
        d.n_voxel[i] = int(geo["n_voxel"][i])
        d.d_voxel[i] = float(geo["d_voxel"][i])
        d.off_origin[i] = float(geo["off_origin"][i])
    for i in range(2):
        d.n_det[i] = int(geo["n_det"][i])
        d.d_det[i] = float(geo["d_det"][i])
        d.off_det[i] = float(geo["off_det"][i])
    d.accuracy = float(geo["accuracy"])
    return d


# ------------------------------------------------------------- the C names

def tigre_geometry_create(geo: dict, angles) -> ctypes.c_void_p:
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    h = ctypes.c_void_p()
    desc = make_desc(geo)
    _check(_lib.tigre_geometry_create(ctypes.byref(desc), ang.ctypes.data_as(_P), len(ang),
                                      ctypes.byref(h)))
    return h


def tigre_geometry_destroy(handle) -> None:
    _check(_lib.tigre_geometry_destroy(handle))


def tigre_forward(handle, vol: torch.Tensor, proj: torch.Tensor, angle_begin: int,
                  angle_count: int, stream=None) -> None:
    vp, vt = _dev(vol, "vol")
    pp, pt = _dev(proj, "proj")
    _check(_lib.tigre_forward(handle, vp, vt, pp, pt, int(angle_begin), int(angle_count),
                              _stream(stream)))


def tigre_backward(handle, proj: torch.Tensor, vol: torch.Tensor, angle_begin: int,
                   angle_count: int, weight="matched", stream=None) -> None:
    pp, pt = _dev(proj, "proj")
    vp, vt = _dev(vol, "vol")
    w = _BP[weight] if isinstance(weight, str) else int(weight)
    _check(_lib.tigre_backward(handle, pp, pt, vp, vt, int(angle_begin), int(angle_count), w,
                               _stream(stream)))


def tigre_tv_step(vol: torch.Tensor, n_steps: int, alpha: float, eps: float,
                  stream=None) -> None:
    vp, vt = _dev(vol, "vol")
    nz, ny, nx = vol.shape
    n = (ctypes.c_int64 * 3)(nx, ny, nz)
    _check(_lib.tigre_tv_step(n, vp, vt, int(n_steps), float(alpha), float(eps),
                              _stream(stream)))


def tigre_tv_step_noalloc(vol: torch.Tensor, n_steps: int, alpha: float, eps: float,
                          stream=None) -> None:
    """tigre_tv_step without device allocation, for callers that must not
    allocate while they run (volumes up to 4,194,304 voxels; calls that
    overlap on the GPU share one scratch area and must not run concurrently)."""
    vp, vt = _dev(vol, "vol")
    nz, ny, nx = vol.shape
    n = (ctypes.c_int64 * 3)(nx, ny, nz)
    _check(_lib.tigre_tv_step_noalloc(n, vp, vt, int(n_steps), float(alpha), float(eps),
                                      _stream(stream)))


def tigre_solver_opts_default() -> tigre_solver_opts:
    o = tigre_solver_opts()
    _check(_lib.tigre_solver_opts_default(ctypes.byref(o)))
    return o


def _solver(fn, handle, proj, vol, opts: tigre_solver_opts, host: bool):
    hist = np.zeros(max(opts.n_iter, 1), dtype=np.float64)
    if proj.dtype != vol.dtype or proj.dtype not in _DTYPES:
        raise TypeError("proj and vol must share one storage dtype (float32/bfloat16/float16)")
    opts.storage = _DTYPES[vol.dtype]
    if host:
        for t, name in ((proj, "proj"), (vol, "vol")):
            if t.is_cuda or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous host tensor")
        opts.flags |= TIGRE_HOST_RESIDENT
        pp, vp = ctypes.c_void_p(proj.data_ptr()), ctypes.c_void_p(vol.data_ptr())
    else:
        pp, _ = _dev(proj, "proj")
        vp, _ = _dev(vol, "vol")
    _check(fn(handle, pp, vp, ctypes.byref(opts), hist.ctypes.data_as(_P)))
    return hist[:opts.n_iter]


def _opts(n_iter, stream, **kw) -> tigre_solver_opts:
    o = tigre_solver_opts_default()
    o.n_iter = int(n_iter)
    o.cuda_stream = _stream(stream).value
    for k, v in kw.items():
        if v is None:
            continue
        if k == "bp_weight" and isinstance(v, str):
            v = _BP[v]
        setattr(o, "lambda_" if k == "lam" else k, v)
    return o


def tigre_sirt(handle, proj, vol, n_iter, lam=1.0, nonneg=False, bp_weight="matched",
               stream=None, host=False) -> np.ndarray:
    o = _opts(n_iter, stream, lam=lam, nonneg=int(nonneg), bp_weight=bp_weight)
    return _solver(_lib.tigre_sirt, handle, proj, vol, o, host)


def tigre_sart(handle, proj, vol, n_iter, subset_size=20, lam=1.0, nonneg=False, tv_steps=0,
               tv_alpha=0.002, tv_eps=1e-8, bp_weight="matched", stream=None,
               host=False) -> np.ndarray:
    o = _opts(n_iter, stream, lam=lam, nonneg=int(nonneg), subset_size=int(subset_size),
              tv_steps=int(tv_steps), tv_alpha=float(tv_alpha), tv_eps=float(tv_eps),
              bp_weight=bp_weight)
    return _solver(_lib.tigre_sart, handle, proj, vol, o, host)


TIGRE_OUT_OF_CORE = 0x4
TIGRE_X0_ZERO = 0x8


def tigre_cgls(handle, proj, vol, n_iter, bp_weight="matched", stream=None,
               host=False, out_of_core=False, device_budget_bytes=0,
               timeout_ms=0, x0_zero=False) -> np.ndarray:
    """CGLS.  host=True stages host tensors through the device; with
    out_of_core=True proj and vol are host tensors, part of the state stays in
    host memory and the volume streams through the GPU in z-slabs; the
    placement and slab thickness follow from device_budget_bytes (0 =
    automatic), see tigre_cgls_ooc_plan.  x0_zero=True: start from x = 0
    without reading vol (r = b, no projection of x0, no upload of x0)."""
    o = _opts(n_iter, stream, bp_weight=bp_weight,
              device_budget_bytes=int(device_budget_bytes), timeout_ms=int(timeout_ms))
    if x0_zero:
        o.flags |= TIGRE_X0_ZERO
    if out_of_core:
        o.flags |= TIGRE_OUT_OF_CORE
        hist = np.zeros(max(n_iter, 1), dtype=np.float64)
        for t, name in ((proj, "proj"), (vol, "vol")):
            if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous float32 host tensor")
        _check(_lib.tigre_cgls(handle, ctypes.c_void_p(proj.data_ptr()),
                               ctypes.c_void_p(vol.data_ptr()), ctypes.byref(o),
                               hist.ctypes.data_as(_P)))
        return hist[:n_iter]
    return _solver(_lib.tigre_cgls, handle, proj, vol, o, host)


def tigre_cgls_ooc_plan(handle, device_budget_bytes: int = 0) -> tuple:
    """(placement, slab planes) of an out-of-core CGLS under the budget:
    placement 2 keeps x, r, q on the device and streams the search direction;
    placement 1 keeps x, p, s in host memory."""
    pl = ctypes.c_int()
    sl = _I64()
    _check(_lib.tigre_cgls_ooc_plan(handle, int(device_budget_bytes), ctypes.byref(pl),
                                    ctypes.byref(sl)))
    return int(pl.value), int(sl.value)


def tigre_cgls_ooc_plan_desc(geo: dict, angles, device_budget_bytes: int) -> tuple:
    """tigre_cgls_ooc_plan from a geometry dict and angles, host only (an
    explicit budget in bytes): (placement, slab planes)."""
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    d = make_desc(geo)
    pl = ctypes.c_int()
    sl = _I64()
    _check(_lib.tigre_cgls_ooc_plan_desc(ctypes.byref(d), ang.ctypes.data_as(_P), ang.size,
                                         int(device_budget_bytes), ctypes.byref(pl),
                                         ctypes.byref(sl)))
    return int(pl.value), int(sl.value)


def tigre_cgls_begin(handle, proj, vol, n_iter_hint=16, bp_weight="matched", stream=None,
                     graph=False, x0_zero=False):
    """Stepwise CGLS; graph=True replays captured iteration pairs as CUDA
    graphs (needs a non-default stream).  proj and vol share one storage
    dtype (float32, bfloat16 or float16); arithmetic is FP32, scalars FP64.
    x0_zero=True zeroes vol and starts from r = b without projecting it."""
    o = _opts(n_iter_hint, stream, bp_weight=bp_weight)
    if graph:
        o.flags |= TIGRE_GRAPH
    if x0_zero:
        o.flags |= TIGRE_X0_ZERO
    pp, pt = _dev(proj, "proj")
    vp, vt = _dev(vol, "vol")
    if pt != vt:
        raise TypeError("proj and vol must share one storage dtype")
    o.storage = vt
    s = ctypes.c_void_p()
    _check(_lib.tigre_cgls_begin(handle, pp, vp, ctypes.byref(o), ctypes.byref(s)))
    return s


def tigre_cgls_iterate(state, n_iter: int) -> None:
    _check(_lib.tigre_cgls_iterate(state, int(n_iter)))


def tigre_cgls_history(state, n: int) -> np.ndarray:
    h = np.zeros(max(n, 1), dtype=np.float64)
    _check(_lib.tigre_cgls_history(state, h.ctypes.data_as(_P), int(n)))
    return h[:n]


def tigre_cgls_end(state) -> None:
    _check(_lib.tigre_cgls_end(state))


def tigre_cgls_batch_begin(handle, projs, vols, n_iter_hint=16, bp_weight="matched", stream=None,
                           graph=False, x0_zero=False):
    """Batched CGLS: len(projs) problems on one geometry handle, iterated
    together (one forward and one backprojection launch per iteration for
    the whole batch).  projs[i] (b) and vols[i] (x0, updated in place) are
    CUDA tensors of one storage dtype; every member's result is bitwise that
    of tigre_cgls on its problem alone."""
    if len(projs) != len(vols) or not projs:
        raise ValueError("need as many volumes as projection sets, at least one")
    o = _opts(n_iter_hint, stream, bp_weight=bp_weight)
    if graph:
        o.flags |= TIGRE_GRAPH
    if x0_zero:
        o.flags |= TIGRE_X0_ZERO
    pps, vps, dts = [], [], set()
    for pr, vo in zip(projs, vols):
        pp, pt = _dev(pr, "proj")
        vp, vt = _dev(vo, "vol")
        pps.append(pp.value)
        vps.append(vp.value)
        dts.update((pt, vt))
    if len(dts) != 1:
        raise TypeError("all projections and volumes must share one storage dtype")
    o.storage = dts.pop()
    parr = (_P * len(pps))(*pps)
    varr = (_P * len(vps))(*vps)
    s = ctypes.c_void_p()
    _check(_lib.tigre_cgls_batch_begin(handle, len(pps), ctypes.cast(parr, _P),
                                       ctypes.cast(varr, _P), ctypes.byref(o), ctypes.byref(s)))
    return s


def tigre_cgls_batch_iterate(state, n_iter: int) -> None:
    _check(_lib.tigre_cgls_batch_iterate(state, int(n_iter)))


def tigre_cgls_batch_history(state, member: int, n: int) -> np.ndarray:
    h = np.zeros(max(n, 1), dtype=np.float64)
    _check(_lib.tigre_cgls_batch_history(state, int(member), h.ctypes.data_as(_P), int(n)))
    return h[:n]


def tigre_cgls_batch_end(state) -> None:
    _check(_lib.tigre_cgls_batch_end(state))


def tigre_cgls_save(state, r_host: torch.Tensor, p_host: torch.Tensor) -> tuple:
    """Copy a stepwise state's residual and search direction into host
    tensors (projection- and volume-shaped, the state's storage dtype);
    returns (gamma, iterations done).  With x these are the whole state."""
    for t, name in ((r_host, "r_host"), (p_host, "p_host")):
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    g = ctypes.c_double()
    n = ctypes.c_int()
    _check(_lib.tigre_cgls_save(state, ctypes.c_void_p(r_host.data_ptr()),
                                r_host.numel() * r_host.element_size(),
                                ctypes.c_void_p(p_host.data_ptr()),
                                p_host.numel() * p_host.element_size(), ctypes.byref(g),
                                ctypes.byref(n)))
    return float(g.value), int(n.value)


def tigre_cgls_resume(handle, proj, vol, r_host, p_host, gamma: float, n_iter_hint=16,
                      bp_weight="matched", stream=None, graph=False):
    """A stepwise state from a checkpoint taken by tigre_cgls_save: vol holds
    the checkpoint's x, proj is b; the iterations continue as the saved
    state's would have."""
    o = _opts(n_iter_hint, stream, bp_weight=bp_weight)
    if graph:
        o.flags |= TIGRE_GRAPH
    pp, pt = _dev(proj, "proj")
    vp, vt = _dev(vol, "vol")
    if pt != vt or r_host.dtype != vol.dtype or p_host.dtype != vol.dtype:
        raise TypeError("proj, vol and the checkpoint must share one storage dtype")
    for t, name in ((r_host, "r_host"), (p_host, "p_host")):
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    if r_host.numel() != proj.numel() or p_host.numel() != vol.numel():
        raise ValueError("checkpoint sizes do not match proj and vol")
    o.storage = vt
    s = ctypes.c_void_p()
    _check(_lib.tigre_cgls_resume(handle, pp, vp, ctypes.c_void_p(r_host.data_ptr()),
                                  r_host.numel() * r_host.element_size(),
                                  ctypes.c_void_p(p_host.data_ptr()),
                                  p_host.numel() * p_host.element_size(), float(gamma),
                                  ctypes.byref(o), ctypes.byref(s)))
    return s


def tigre_forward_samples(handle, angle_begin: int, angle_count: int) -> int:
    n = _I64()
    _check(_lib.tigre_forward_samples(handle, int(angle_begin), int(angle_count), ctypes.byref(n)))
    return int(n.value)


def _host_f32(t: torch.Tensor, name: str):
    if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 host tensor")
    return ctypes.c_void_p(t.data_ptr())


def tigre_forward_ooc(handle, vol_host: torch.Tensor, proj: torch.Tensor, angle_begin: int,
                      angle_count: int, slab_planes: int = 0, stream=None) -> None:
    """Out-of-core A x: host volume streamed in z-slabs, device projections."""
    pp, pt = _dev(proj, "proj")
    if pt != TIGRE_F32:
        raise TypeError("proj must be float32")
    _check(_lib.tigre_forward_ooc(handle, _host_f32(vol_host, "vol_host"), pp, int(angle_begin),
                                  int(angle_count), int(slab_planes), _stream(stream)))


def tigre_backward_ooc(handle, proj: torch.Tensor, vol_host: torch.Tensor, angle_begin: int,
                       angle_count: int, weight="matched", slab_planes: int = 0,
                       angle_chunk: int = 0, stream=None) -> None:
    """Out-of-core A^T y into a host volume; proj on device or host."""
    on_host = not proj.is_cuda
    pp = _host_f32(proj, "proj") if on_host else _dev(proj, "proj")[0]
    w = _BP[weight] if isinstance(weight, str) else int(weight)
    _check(_lib.tigre_backward_ooc(handle, pp, int(on_host), _host_f32(vol_host, "vol_host"),
                                   int(angle_begin), int(angle_count), w, int(slab_planes),
                                   int(angle_chunk), _stream(stream)))


FWD_AUTO, FWD_L1, FWD_TMA, FWD_QUAD, FWD_QUAD_PAIR = 0, 1, 2, 3, 4
FWD_QUAD_ANGLES2, FWD_QUAD_ANGLES4 = 5, 6  # warps of 16 pixels x 2 angles / 8 x 4


def tigre_forward_angle_groups(geo: dict, angles, size: int = 2):
    """The forward projector's angle groups (host only): (table of shape
    (n_groups, size) with -1 filling short groups, drift in voxels, whether
    the automatic path pairs angles)."""
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    d = make_desc(geo)
    ng, drift, auto = _I64(), ctypes.c_double(), ctypes.c_int()
    _check(_lib.tigre_forward_angle_groups(ctypes.byref(d), ang.ctypes.data_as(_P), ang.size,
                                           int(size), None, 0, ctypes.byref(ng),
                                           ctypes.byref(drift), ctypes.byref(auto)))
    tab = np.zeros(ng.value * size, dtype=np.int32)
    _check(_lib.tigre_forward_angle_groups(ctypes.byref(d), ang.ctypes.data_as(_P), ang.size,
                                           int(size), tab.ctypes.data_as(_P), tab.size,
                                           ctypes.byref(ng), ctypes.byref(drift),
                                           ctypes.byref(auto)))
    return tab.reshape(-1, size), float(drift.value), bool(auto.value)


def tigre_fdk(handle, proj: torch.Tensor, vol: torch.Tensor, stream=None) -> None:
    """FDK reconstruction of all the handle's angles into vol (device)."""
    pp, pt = _dev(proj, "proj")
    vp, vt = _dev(vol, "vol")
    _check(_lib.tigre_fdk(handle, pp, pt, vp, vt, _stream(stream)))


def tigre_rof_denoise(f: torch.Tensor, lam: float, n_iter: int, out: torch.Tensor = None,
                      stream=None) -> torch.Tensor:
    """ROF-model TV minimisation of a device F32 volume (out may be f)."""
    fp, ft = _dev(f, "f")
    if ft != TIGRE_F32:
        raise TypeError("f must be float32")
    if out is None:
        out = torch.empty_like(f)
    op, ot = _dev(out, "out")
    if ot != TIGRE_F32 or out.shape != f.shape:
        raise TypeError("out must be a float32 tensor of f's shape")
    n = (ctypes.c_int64 * 3)(f.shape[2], f.shape[1], f.shape[0])
    _check(_lib.tigre_rof_denoise(n, fp, op, float(lam), int(n_iter), _stream(stream)))
    return out


def tigre_tv_step_ooc(vol_host: torch.Tensor, n_steps: int, alpha: float, eps: float = 1e-8,
                      slab_planes: int = 0, halo_depth: int = 1, stream=None) -> None:
    """Out-of-core TV steps on a host F32 volume (in place): z-slabs with
    halo buffers and the per-slab norm approximation."""
    n = (ctypes.c_int64 * 3)(vol_host.shape[2], vol_host.shape[1], vol_host.shape[0])
    _check(_lib.tigre_tv_step_ooc(n, _host_f32(vol_host, "vol_host"), int(n_steps), float(alpha),
                                  float(eps), int(slab_planes), int(halo_depth), _stream(stream)))


_allocator_refs = None  # keeps the installed ctypes callbacks alive


def tigre_set_allocator(alloc=None, free=None) -> None:
    """Install Python callables as the library's device workspace allocator:
    alloc(nbytes, stream_ptr) -> device pointer (int, 0 on failure) and
    free(ptr, stream_ptr); None, None restores the CUDA default.  Only while
    no Geometry or CGLS state is alive."""
    global _allocator_refs
    if alloc is None and free is None:
        _check(_lib.tigre_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _allocator_refs = None
        return

    def _a(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(stream or 0)) or 0)
        except Exception:
            return 0

    def _f(ptr, stream, ctx):
        try:
            free(int(ptr), int(stream or 0))
        except Exception:
            pass

    refs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(_lib.tigre_set_allocator(refs[0], refs[1], None))
    _allocator_refs = refs


def use_torch_allocator(on: bool = True) -> None:
    """Route the library's device workspaces through PyTorch's caching
    allocator (on the stream the library names, the current device), so the
    library and the framework share one memory pool."""
    if not on:
        tigre_set_allocator(None, None)
        return

    def _alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device=torch.cuda.current_device(),
                                                  stream=stream)

    def _free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    tigre_set_allocator(_alloc, _free)


PROJ_INTERPOLATED, PROJ_SIDDON = 0, 1


def tigre_geometry_set_projector(handle, projector) -> None:
    """'interpolated' (default) or 'siddon' (or the PROJ_* value)."""
    if isinstance(projector, str):
        projector = {"interpolated": PROJ_INTERPOLATED, "siddon": PROJ_SIDDON}[projector]
    _check(_lib.tigre_geometry_set_projector(handle, int(projector)))


def tigre_geometry_set_brick(handle, edge: int) -> None:
    """x-y brick edge (voxels) of out-of-core slab projections; 0 = default."""
    _check(_lib.tigre_geometry_set_brick(handle, int(edge)))


def tigre_geometry_set_forward_path(handle, path: int) -> None:
    _check(_lib.tigre_geometry_set_forward_path(handle, int(path)))


def tigre_geometry_error_flags(handle, clear: bool = True) -> int:
    f = ctypes.c_int()
    _check(_lib.tigre_geometry_error_flags(handle, ctypes.byref(f), int(bool(clear))))
    return int(f.value)


def tigre_profile_enable(on: bool = True) -> None:
    _check(_lib.tigre_profile_enable(int(bool(on))))


def tigre_profile_read(kind: int):
    """(number of timed calls, total device ms) for a kernel class."""
    n, ms = _I64(), ctypes.c_double()
    _check(_lib.tigre_profile_read(int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def tigre_launch_count() -> int:
    return int(_lib.tigre_launch_count())


# ------------------------------------------------------------ convenience

class Geometry:
    """Owns a geometry handle; shapes of its volume and projections."""

    def __init__(self, geo: dict, angles):
        self.geo = dict(geo)
        self.angles = np.ascontiguousarray(angles, dtype=np.float64)
        self.handle = tigre_geometry_create(self.geo, self.angles)
        nx, ny, nz = self.geo["n_voxel"]
        nu, nv = self.geo["n_det"]
        self.vol_shape = (nz, ny, nx)
        self.proj_shape = (len(self.angles), nv, nu)

    def close(self):
        if self.handle is not None:
            tigre_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def forward(self, vol, out=None, angle_begin=0, angle_count=None, dtype=None, stream=None):
        na = len(self.angles) - angle_begin if angle_count is None else angle_count
        if out is None:
            out = torch.empty((na,) + self.proj_shape[1:], device=vol.device,
                              dtype=dtype or vol.dtype)
        tigre_forward(self.handle, vol, out, angle_begin, na, stream)
        return out

    def fdk(self, proj, out=None, dtype=None, stream=None):
        if out is None:
            out = torch.empty(self.vol_shape, device=proj.device, dtype=dtype or proj.dtype)
        tigre_fdk(self.handle, proj, out, stream)
        return out

    def backward(self, proj, out=None, angle_begin=0, weight="matched", dtype=None, stream=None):
        na = proj.shape[0]
        if out is None:
            out = torch.empty(self.vol_shape, device=proj.device, dtype=dtype or proj.dtype)
        tigre_backward(self.handle, proj, out, angle_begin, na, weight, stream)
        return out
