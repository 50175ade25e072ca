"""Independent reference computations used to pin the oracle.

Nothing here calls the oracle or the CUDA library.  Each function reaches a
quantity the oracle must agree with by a different route:

* ``exact_ray_integral``: the exact line integral of the trilinear
  interpolant, splitting the ray at every voxel-centre plane it crosses and
  integrating each piece (a cubic in t) with 2-point Gauss-Legendre.
* ``ellipsoid_chord``: analytic chord length of a ray through an ellipsoid.
* ``detector_hit``: detector coordinates of a point, from intersecting the
  line source->point with the detector plane (vector algebra, not the
  magnification formula the oracle uses).
"""
from __future__ import annotations

import numpy as np


def rot_z(theta: float) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def frame(geo: dict, theta: float):
    """Source, detector centre, e_u, e_v by rotating the theta=0 frame."""
    R = rot_z(theta)
    S = R @ np.array([geo["DSO"], 0.0, 0.0])
    D = R @ np.array([-(geo["DSD"] - geo["DSO"]), 0.0, 0.0])
    eu = R @ np.array([0.0, 1.0, 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    return S, D, eu, ev


def pixel_centre(geo: dict, theta: float, p: float, q: float) -> np.ndarray:
    S, D, eu, ev = frame(geo, theta)
    nu, nv = geo["n_det"]
    du, dv = geo["d_det"]
    u = (p - (nu - 1) / 2.0) * du + geo["off_det"][0]
    v = (q - (nv - 1) / 2.0) * dv + geo["off_det"][1]
    return D + u * eu + v * ev


def world_to_index(geo: dict, X: np.ndarray) -> np.ndarray:
    n = np.array(geo["n_voxel"], dtype=float)
    d = np.array(geo["d_voxel"])
    o = np.array(geo["off_origin"])
    return (X - o) / d + (n - 1) / 2.0


def trilinear_padded(vol: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of vol (nz, ny, nx) at index points (m, 3) as
    (x, y, z), using an explicitly zero-padded copy of the volume."""
    pad = np.pad(np.asarray(vol, dtype=np.float64), 1)
    out = np.zeros(len(pts))
    base = np.floor(pts).astype(np.int64)
    frac = pts - base
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                ix = base[:, 0] + bx + 1
                iy = base[:, 1] + by + 1
                iz = base[:, 2] + bz + 1
                ok = ((ix >= 0) & (iy >= 0) & (iz >= 0) & (ix < pad.shape[2]) &
                      (iy < pad.shape[1]) & (iz < pad.shape[0]))
                w = (np.where(bx, frac[:, 0], 1 - frac[:, 0]) *
                     np.where(by, frac[:, 1], 1 - frac[:, 1]) *
                     np.where(bz, frac[:, 2], 1 - frac[:, 2]))
                val = np.zeros(len(pts))
                val[ok] = pad[iz[ok], iy[ok], ix[ok]]
                out += w * val
    return out


def exact_ray_integral(geo: dict, vol: np.ndarray, theta: float, p: int, q: int) -> float:
    """Exact integral (mm x density) of the trilinear interpolant along the
    ray from the source to pixel (p, q)."""
    S, _, _, _ = frame(geo, theta)
    P = pixel_centre(geo, theta, p, q)
    xs = world_to_index(geo, S)
    xp = world_to_index(geo, P)
    r = xp - xs
    n = np.array(geo["n_voxel"], dtype=float)
    seg = np.linalg.norm(P - S)
    lo, hi = 0.0, 1.0
    for a in range(3):
        if r[a] == 0.0:
            if not (-1.0 < xs[a] < n[a]):
                return 0.0
            continue
        t1, t2 = sorted(((-1.0 - xs[a]) / r[a], (n[a] - xs[a]) / r[a]))
        lo, hi = max(lo, t1), min(hi, t2)
    if hi <= lo:
        return 0.0
    cuts = [lo, hi]
    for a in range(3):
        if r[a] == 0.0:
            continue
        ka = np.arange(np.ceil(min(xs[a] + lo * r[a], xs[a] + hi * r[a])),
                       np.floor(max(xs[a] + lo * r[a], xs[a] + hi * r[a])) + 1)
        cuts.extend(((ka - xs[a]) / r[a]).tolist())
    cuts = np.unique(np.clip(np.array(cuts), lo, hi))
    a_, b_ = cuts[:-1], cuts[1:]
    mid, half = 0.5 * (a_ + b_), 0.5 * (b_ - a_)
    g = 1.0 / np.sqrt(3.0)
    total = 0.0
    for node in (-g, g):
        t = mid + node * half
        pts = xs[None, :] + t[:, None] * r[None, :]
        total += np.sum(half * trilinear_padded(vol, pts))
    return float(total * seg)


def ellipsoid_chord(S: np.ndarray, P: np.ndarray, centre, axes, rot) -> float:
    """Length (mm) of the part of segment S->P inside the ellipsoid whose
    axis a points along column a of rot with semi-axis axes[a]."""
    M = np.asarray(rot).T / np.asarray(axes)[:, None]
    y0 = M @ (S - np.asarray(centre))
    y1 = M @ (P - S)
    A = y1 @ y1
    B = 2.0 * (y0 @ y1)
    C = y0 @ y0 - 1.0
    disc = B * B - 4 * A * C
    if disc <= 0:
        return 0.0
    sq = np.sqrt(disc)
    t1, t2 = (-B - sq) / (2 * A), (-B + sq) / (2 * A)
    t1, t2 = max(t1, 0.0), min(t2, 1.0)
    return max(t2 - t1, 0.0) * float(np.linalg.norm(P - S))


def detector_hit(geo: dict, theta: float, X: np.ndarray):
    """Fractional pixel indices (p, q) where the line source->X meets the
    detector plane, and the distance along the central axis source->X."""
    S, D, eu, ev = frame(geo, theta)
    c = (D - S) / np.linalg.norm(D - S)
    depth = (X - S) @ c
    lam = ((D - S) @ c) / depth
    Pt = S + lam * (X - S)
    u = (Pt - D) @ eu
    v = (Pt - D) @ ev
    nu, nv = geo["n_det"]
    du, dv = geo["d_det"]
    p = (u - geo["off_det"][0]) / du + (nu - 1) / 2.0
    q = (v - geo["off_det"][1]) / dv + (nv - 1) / 2.0
    return p, q, depth


def voxel_centre(geo: dict, i, j, k) -> np.ndarray:
    n = np.array(geo["n_voxel"], dtype=float)
    d = np.array(geo["d_voxel"])
    o = np.array(geo["off_origin"])
    return (np.array([i, j, k], dtype=float) - (n - 1) / 2.0) * d + o


def box_chord(S: np.ndarray, P: np.ndarray, lo, hi) -> float:
    """Length (mm) of the part of segment S->P inside the world-space box
    [lo, hi] (Kay-Kajiya slab clipping in world coordinates)."""
    d = P - S
    t0, t1 = 0.0, 1.0
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] < S[a] < hi[a]):
                return 0.0
            continue
        ta, tb = sorted(((lo[a] - S[a]) / d[a], (hi[a] - S[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def voxel_box(geo: dict, i: int, j: int, k: int):
    """World-space box of voxel (i, j, k): its centre +- half a voxel."""
    n = np.array(geo["n_voxel"], dtype=float)
    d = np.array(geo["d_voxel"])
    o = np.array(geo["off_origin"])
    c = (np.array([i, j, k], dtype=float) - (n - 1) / 2.0) * d + o
    return c - d / 2.0, c + d / 2.0


def volume_box(geo: dict):
    """World-space box covered by all voxels."""
    n = np.array(geo["n_voxel"], dtype=float)
    d = np.array(geo["d_voxel"])
    o = np.array(geo["off_origin"])
    return o - n * d / 2.0, o + n * d / 2.0
