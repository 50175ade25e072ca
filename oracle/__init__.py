"""FP64 CPU oracle for the cone-beam CT hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1905_03748_gb300``) and never imports it.

Operators (``oracle.c``, plain C, FP64, OpenMP over independent rays/voxels):
    forward, forward_rays          interpolated ray-driven projector (Sec. 2.1)
    backward, backward_voxels      voxel-driven BP, FDK / matched weights (Sec. 2.2)
    adjoint, adjoint_voxels        exact transpose of the projector
    siddon_forward, siddon_forward_rays, siddon_adjoint
                                   ray-voxel intersection (Siddon) projector
    tv_value, tv_grad, tv_steps    gradient-descent TV (Sec. 2.3)
    tv_steps_split (this file)     the same steps on z-slabs with halo buffers and
                                   the per-slab norm approximation (Sec. 2.3)
    rof_denoise (this file)        ROF-model TV minimisation (Sec. 2.3), first-order
                                   primal-dual iteration
    ramp_kernel, fdk               FDK: cosine weights, Ram-Lak ramp filter
                                   along detector rows, FDK-weighted backprojection
Solvers (this file, numpy FP64, written as the textbook iterations):
    sirt, os_sart (with optional TV after each iteration), cgls.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BP_MATCHED = 0
BP_FDK = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int64
            sig = {
                "oracle_forward": [P, P, I, P, P],
                "oracle_forward_rays": [P, P, P, P, I, P],
                "oracle_sample_count": [P, P, I],
                "oracle_ray_params": [P, P, P, I, P],
                "oracle_backward": [P, P, I, P, P, ctypes.c_int],
                "oracle_backward_voxels": [P, P, I, P, P, I, P, ctypes.c_int],
                "oracle_adjoint": [P, P, I, P, P],
                "oracle_adjoint_voxels": [P, P, I, P, P, I, P],
                "oracle_siddon_forward": [P, P, I, P, P],
                "oracle_siddon_forward_rays": [P, P, P, P, I, P],
                "oracle_siddon_adjoint": [P, P, I, P, P],
                "oracle_tv_value": [P, I, I, I, ctypes.c_double],
                "oracle_tv_grad": [P, I, I, I, ctypes.c_double, P],
                "oracle_tv_grad_voxels": [P, I, I, I, ctypes.c_double, P, I, P],
                "oracle_tv_steps": [P, I, I, I, ctypes.c_int, ctypes.c_double, ctypes.c_double],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = None
            lib.oracle_sample_count.restype = ctypes.c_int64
            lib.oracle_tv_value.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _geo_array(geo: dict) -> np.ndarray:
    return np.array([geo["DSO"], geo["DSD"], *geo["n_voxel"], *geo["d_voxel"],
                     *geo["off_origin"], *geo["n_det"], *geo["d_det"], *geo["off_det"],
                     geo["accuracy"]], dtype=np.float64)


def _shapes(geo):
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    return (nz, ny, nx), (nv, nu)


# ----------------------------------------------------------------- operators

def forward(geo: dict, angles, vol) -> np.ndarray:
    """A x: proj (A, nv, nu) from vol (nz, ny, nx)."""
    lib = _load()
    vshape, dshape = _shapes(geo)
    ang = _f64(angles)
    v = _f64(vol).reshape(vshape)
    out = np.empty((len(ang),) + dshape, dtype=np.float64)
    lib.oracle_forward(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(v), _ptr(out))
    return out


def forward_rays(geo: dict, angles, vol, rays) -> np.ndarray:
    """A x at selected rays given as (a, q, p) rows."""
    lib = _load()
    vshape, _ = _shapes(geo)
    v = _f64(vol).reshape(vshape)
    idx = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    lib.oracle_forward_rays(_ptr(_geo_array(geo)), _ptr(_f64(angles)), _ptr(v), _ptr(idx),
                            len(idx), _ptr(out))
    return out


def sample_count(geo: dict, angles) -> int:
    """Total quadrature samples of one forward projection (sum of K)."""
    ang = _f64(angles)
    return int(_load().oracle_sample_count(_ptr(_geo_array(geo)), _ptr(ang), len(ang)))


def ray_params(geo: dict, angles, rays) -> np.ndarray:
    """(K, len_mm, t_in, t_out) per selected ray; zeros for rays that miss."""
    idx = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty((len(idx), 4), dtype=np.float64)
    _load().oracle_ray_params(_ptr(_geo_array(geo)), _ptr(_f64(angles)), _ptr(idx), len(idx),
                              _ptr(out))
    return out


def backward(geo: dict, angles, proj, mode: int = BP_MATCHED) -> np.ndarray:
    """Voxel-driven weighted backprojection (mode BP_MATCHED or BP_FDK)."""
    lib = _load()
    vshape, dshape = _shapes(geo)
    ang = _f64(angles)
    p = _f64(proj).reshape((len(ang),) + dshape)
    out = np.empty(vshape, dtype=np.float64)
    lib.oracle_backward(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(p), _ptr(out), int(mode))
    return out


def backward_voxels(geo: dict, angles, proj, voxels, mode: int = BP_MATCHED) -> np.ndarray:
    """Backprojection at selected voxels given as (i, j, k) rows."""
    lib = _load()
    _, dshape = _shapes(geo)
    ang = _f64(angles)
    p = _f64(proj).reshape((len(ang),) + dshape)
    idx = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    lib.oracle_backward_voxels(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(p), _ptr(idx),
                               len(idx), _ptr(out), int(mode))
    return out


def siddon_forward(geo: dict, angles, vol) -> np.ndarray:
    """Ray-voxel intersection projection of a piecewise-constant volume."""
    lib = _load()
    vshape, dshape = _shapes(geo)
    ang = _f64(angles)
    v = _f64(vol).reshape(vshape)
    out = np.empty((len(ang),) + dshape, dtype=np.float64)
    lib.oracle_siddon_forward(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(v), _ptr(out))
    return out


def siddon_forward_rays(geo: dict, angles, vol, rays) -> np.ndarray:
    """Siddon projection at selected rays given as (a, q, p) rows."""
    lib = _load()
    vshape, _ = _shapes(geo)
    v = _f64(vol).reshape(vshape)
    idx = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    lib.oracle_siddon_forward_rays(_ptr(_geo_array(geo)), _ptr(_f64(angles)), _ptr(v), _ptr(idx),
                                   len(idx), _ptr(out))
    return out


def siddon_adjoint(geo: dict, angles, proj) -> np.ndarray:
    """Exact transpose of siddon_forward (serial scatter)."""
    lib = _load()
    vshape, dshape = _shapes(geo)
    ang = _f64(angles)
    p = _f64(proj).reshape((len(ang),) + dshape)
    out = np.empty(vshape, dtype=np.float64)
    lib.oracle_siddon_adjoint(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(p), _ptr(out))
    return out


def adjoint(geo: dict, angles, proj) -> np.ndarray:
    """Exact transpose of forward (serial scatter)."""
    lib = _load()
    vshape, dshape = _shapes(geo)
    ang = _f64(angles)
    p = _f64(proj).reshape((len(ang),) + dshape)
    out = np.empty(vshape, dtype=np.float64)
    lib.oracle_adjoint(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(p), _ptr(out))
    return out


def adjoint_voxels(geo: dict, angles, proj, voxels) -> np.ndarray:
    """Exact transpose of forward evaluated at selected voxels."""
    lib = _load()
    _, dshape = _shapes(geo)
    ang = _f64(angles)
    p = _f64(proj).reshape((len(ang),) + dshape)
    idx = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    lib.oracle_adjoint_voxels(_ptr(_geo_array(geo)), _ptr(ang), len(ang), _ptr(p), _ptr(idx),
                              len(idx), _ptr(out))
    return out


def ramp_kernel(n: int) -> np.ndarray:
    """Dimensionless Ram-Lak kernel h[k], k = -(n-1) .. n-1: the coefficients
    of the ramp |w| band-limited to the Nyquist frequency (Kak & Slaney's
    discrete ramp), h[0] = 1/4, h[odd k] = -1/(pi k)^2, h[even k] = 0.  With
    sample spacing tau the kernel is h / tau^2."""
    k = np.arange(-(n - 1), n, dtype=np.float64)
    h = np.zeros_like(k)
    h[k == 0] = 0.25
    odd = (np.abs(k) % 2) == 1
    h[odd] = -1.0 / (np.pi * k[odd]) ** 2
    return h


def fdk_angle_weights(angles) -> np.ndarray:
    """Angular quadrature weight of each angle: half the angle between its
    neighbours on the circle (2 pi / N for N uniform angles)."""
    a = np.mod(_f64(angles), 2 * np.pi)
    order = np.argsort(a)
    srt = a[order]
    nxt = np.roll(srt, -1)
    prv = np.roll(srt, 1)
    gap_n = np.mod(nxt - srt, 2 * np.pi)
    gap_p = np.mod(srt - prv, 2 * np.pi)
    if len(a) == 1:
        gap_n = gap_p = np.array([2 * np.pi])
    w = np.empty_like(a)
    w[order] = 0.5 * (gap_n + gap_p)
    return w


def fdk(geo: dict, angles, proj) -> np.ndarray:
    """Feldkamp-Davis-Kress reconstruction of a full circular scan:
    each projection is weighted by DSD/sqrt(DSD^2 + u^2 + v^2), each detector
    row is convolved (linearly, zero outside the detector) with the Ram-Lak
    kernel of the detector pitch scaled to the isocentre (du DSO/DSD), and the
    filtered projections are backprojected with the FDK distance weight
    (DSO/(DSO-s))^2, each angle times half its angular weight."""
    _, dshape = _shapes(geo)
    ang = _f64(angles)
    g = _f64(proj).reshape((len(ang),) + dshape)
    nu, nv = geo["n_det"]
    du, dv = geo["d_det"]
    u = (np.arange(nu) - (nu - 1) / 2.0) * du + geo["off_det"][0]
    v = (np.arange(nv) - (nv - 1) / 2.0) * dv + geo["off_det"][1]
    dsd = geo["DSD"]
    cosw = dsd / np.sqrt(dsd ** 2 + u[None, :] ** 2 + v[:, None] ** 2)
    tau = du * geo["DSO"] / dsd
    h = ramp_kernel(nu) / tau
    q = np.empty_like(g)
    for a in range(len(ang)):
        gw = g[a] * cosw
        for r in range(nv):
            q[a, r] = np.convolve(gw[r], h)[nu - 1:2 * nu - 1]
    q *= 0.5 * fdk_angle_weights(ang)[:, None, None]
    return backward(geo, ang, q, BP_FDK)


def tv_value(vol, eps: float) -> float:
    v = _f64(vol)
    nz, ny, nx = v.shape
    return float(_load().oracle_tv_value(_ptr(v), nx, ny, nz, float(eps)))


def tv_grad(vol, eps: float) -> np.ndarray:
    v = _f64(vol)
    nz, ny, nx = v.shape
    g = np.empty_like(v)
    _load().oracle_tv_grad(_ptr(v), nx, ny, nz, float(eps), _ptr(g))
    return g


def tv_grad_voxels(vol, eps: float, voxels) -> np.ndarray:
    v = _f64(vol)
    nz, ny, nx = v.shape
    idx = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    _load().oracle_tv_grad_voxels(_ptr(v), nx, ny, nz, float(eps), _ptr(idx), len(idx), _ptr(out))
    return out


def tv_steps(vol, n_steps: int, alpha: float, eps: float) -> np.ndarray:
    """n_steps of x <- x - alpha g/||g|| (Sec. 2.3 gradient descent)."""
    v = _f64(vol).copy()
    nz, ny, nx = v.shape
    _load().oracle_tv_steps(_ptr(v), nx, ny, nz, int(n_steps), float(alpha), float(eps))
    return v


# ------------------------------------------------------------------- solvers

def tv_steps_split(vol, n_steps: int, alpha: float, eps: float, slab: int, depth: int,
                   halo: int = None) -> np.ndarray:
    """Gradient-descent TV on z-slabs, the paper's splitting of a regulariser
    (Sec. 2.3): in rounds of k = min(depth, steps left) steps, every slab takes
    its k steps on its own, from the previous round's values, with k planes of
    those values on each side as a buffer (a buffer as deep as the number of
    independent steps); the norm of the update is approximated from the
    slab's own voxels as if uniformly distributed over the volume,
    ||g|| ~ ||g_slab|| sqrt(N / N_slab); the slab's own planes are then
    written back.  halo overrides the buffer depth (for tests)."""
    f = _f64(vol).copy()
    nz = f.shape[0]
    N = f.size
    plane = f.shape[1] * f.shape[2]
    done = 0
    while done < n_steps:
        k = min(depth, n_steps - done)
        h = k if halo is None else halo
        old = f.copy()
        for z0 in range(0, nz, slab):
            z1 = min(nz, z0 + slab)
            lo, hi = max(0, z0 - h), min(nz, z1 + h)
            sub = old[lo:hi].copy()
            scale = np.sqrt(N / ((z1 - z0) * plane))
            for _ in range(k):
                g = tv_grad(sub, eps)
                nrm = np.sqrt(np.sum(g[z0 - lo:z1 - lo] ** 2)) * scale
                if nrm > 0:
                    sub = sub - alpha * g / nrm
            f[z0:z1] = sub[z0 - lo:z1 - lo]
        done += k
    return f


def rof_grad(u):
    """Forward differences along x, y, z of u (nz, ny, nx); zero at the last
    index of each axis (Neumann boundary).  Returns (gx, gy, gz)."""
    u = _f64(u)
    gx, gy, gz = np.zeros_like(u), np.zeros_like(u), np.zeros_like(u)
    gx[:, :, :-1] = u[:, :, 1:] - u[:, :, :-1]
    gy[:, :-1, :] = u[:, 1:, :] - u[:, :-1, :]
    gz[:-1, :, :] = u[1:, :, :] - u[:-1, :, :]
    return gx, gy, gz


def rof_div(px, py, pz):
    """Divergence, the negative adjoint of rof_grad: <grad u, p> = -<u, div p>."""
    d = np.zeros_like(px)
    for p_, ax in ((px, 2), (py, 1), (pz, 0)):
        p_ = np.moveaxis(p_, ax, 0)
        dd = np.moveaxis(d, ax, 0)
        n = p_.shape[0]
        if n == 1:
            continue
        dd[0] += p_[0]
        dd[1:n - 1] += p_[1:n - 1] - p_[0:n - 2]
        dd[n - 1] -= p_[n - 2]
    return d


def rof_denoise(f, lam: float, n_iter: int) -> np.ndarray:
    """ROF model min_u ||grad u||_(2,1) + lam/2 ||u - f||^2 (isotropic TV),
    solved with the first-order primal-dual iteration (over-relaxation 1,
    step sizes tau = sigma = 1/sqrt(12), the bound ||grad||^2 <= 12 in 3-D):
        p    <- (p + sigma grad(ubar)) / max(1, |p + sigma grad(ubar)|)
        u'   <- (u + tau div p + tau lam f) / (1 + tau lam)
        ubar <- 2 u' - u,  u <- u'
    from u = ubar = f, p = 0."""
    f = _f64(f)
    tau = sigma = 1.0 / np.sqrt(12.0)
    u = f.copy()
    ubar = f.copy()
    px, py, pz = np.zeros_like(f), np.zeros_like(f), np.zeros_like(f)
    for _ in range(n_iter):
        gx, gy, gz = rof_grad(ubar)
        px, py, pz = px + sigma * gx, py + sigma * gy, pz + sigma * gz
        nrm = np.maximum(1.0, np.sqrt(px * px + py * py + pz * pz))
        px, py, pz = px / nrm, py / nrm, pz / nrm
        un = (u + tau * rof_div(px, py, pz) + tau * lam * f) / (1.0 + tau * lam)
        ubar = 2.0 * un - u
        u = un
    return u


def rof_objective(u, f, lam: float) -> float:
    gx, gy, gz = rof_grad(u)
    return float(np.sum(np.sqrt(gx * gx + gy * gy + gz * gz)) +
                 0.5 * lam * np.sum((_f64(u) - _f64(f)) ** 2))


def _guarded_reciprocal(a: np.ndarray, floor: float = 1e-12) -> np.ndarray:
    out = np.zeros_like(a)
    np.divide(1.0, a, out=out, where=a > floor)
    return out


def sirt(geo, angles, b, n_iter, lam=1.0, nonneg=False, x0=None, mode=BP_MATCHED):
    """SIRT: x <- x + lam V A^T W (b - A x), W = 1/(A 1), V = 1/(A^T 1).

    Returns (x, resid) with resid[k] = ||b - A x_k||_2 before update k.
    """
    vshape, _ = _shapes(geo)
    b = _f64(b)
    x = np.zeros(vshape) if x0 is None else _f64(x0).reshape(vshape).copy()
    W = _guarded_reciprocal(forward(geo, angles, np.ones(vshape)))
    V = _guarded_reciprocal(backward(geo, angles, np.ones(b.shape), mode))
    resid = []
    for _ in range(n_iter):
        r = b - forward(geo, angles, x)
        resid.append(float(np.linalg.norm(r)))
        x = x + lam * V * backward(geo, angles, W * r, mode)
        if nonneg:
            x = np.maximum(x, 0.0)
    return x, np.array(resid)


def os_sart(geo, angles, b, n_iter, subset=20, lam=1.0, nonneg=False, x0=None,
            tv_steps_n=0, tv_alpha=0.002, tv_eps=1e-8, mode=BP_MATCHED):
    """OS-SART over contiguous subsets of `subset` angles, visited in order;
    optional gradient-descent TV after each full iteration with step
    alpha * ||x_after_data - x_before_data||_2.

    Returns (x, resid) with resid[k] = sqrt(sum_s ||b_s - A_s x||^2) over the
    subset residuals computed during iteration k.
    """
    vshape, _ = _shapes(geo)
    ang = _f64(angles)
    b = _f64(b)
    x = np.zeros(vshape) if x0 is None else _f64(x0).reshape(vshape).copy()
    blocks = [np.arange(s, min(s + subset, len(ang))) for s in range(0, len(ang), subset)]
    Ws, Vs = [], []
    for blk in blocks:
        Ws.append(_guarded_reciprocal(forward(geo, ang[blk], np.ones(vshape))))
        Vs.append(_guarded_reciprocal(backward(geo, ang[blk], np.ones((len(blk),) + b.shape[1:]),
                                               mode)))
    resid = []
    for _ in range(n_iter):
        x_prev = x.copy()
        rr = 0.0
        for blk, W, V in zip(blocks, Ws, Vs):
            r = b[blk] - forward(geo, ang[blk], x)
            rr += float(np.sum(r * r))
            x = x + lam * V * backward(geo, ang[blk], W * r, mode)
            if nonneg:
                x = np.maximum(x, 0.0)
        resid.append(np.sqrt(rr))
        if tv_steps_n > 0:
            step = tv_alpha * float(np.linalg.norm(x - x_prev))
            x = tv_steps(x, tv_steps_n, step, tv_eps)
    return x, np.array(resid)


def cgls(geo, angles, b, n_iter, x0=None, bp="matched", projector="interpolated"):
    """CGLS (conjugate gradients on A^T A x = A^T b), FP64 scalars.

    bp = "matched" (voxel-driven pseudo-matched backprojector) or "adjoint"
    (exact transpose of the projector); projector = "interpolated" or
    "siddon".  Returns (x, resid) with resid[k] = ||r_k||_2 after iteration k.
    """
    vshape, _ = _shapes(geo)
    b = _f64(b)
    A = (lambda v: siddon_forward(geo, angles, v)) if projector == "siddon" else \
        (lambda v: forward(geo, angles, v))
    if bp == "adjoint":
        At = (lambda y: siddon_adjoint(geo, angles, y)) if projector == "siddon" else \
            (lambda y: adjoint(geo, angles, y))
    else:
        At = lambda y: backward(geo, angles, y, BP_MATCHED)  # noqa: E731
    x = np.zeros(vshape) if x0 is None else _f64(x0).reshape(vshape).copy()
    r = b - A(x) if x0 is not None else b.copy()
    p = At(r)
    gamma = float(np.sum(p * p))
    resid = []
    for _ in range(n_iter):
        q = A(p)
        alpha = gamma / float(np.sum(q * q))
        x = x + alpha * p
        r = r - alpha * q
        resid.append(float(np.linalg.norm(r)))
        s = At(r)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x, np.array(resid)
