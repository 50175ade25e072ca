"""Seeded synthetic inputs: geometries, angle sets, ellipsoid phantoms, noise.

This module holds no projector, backprojector, regulariser or solver
arithmetic.  It only builds the inputs that both the CUDA path and the CPU
oracle consume, so both sides see byte-identical data.

Workload recipe (the paper's experiments use N^3 volumes, N^2 detectors and N
angles on a circular cone-beam orbit, Sec. 3.1; its scans are not available,
so seeded phantoms stand in for them):

* DSO = 1000 mm, DSD = 1536 mm for every workload.
* Voxel size keeps a 256 mm field of view unless a workload fixes it.
* Detector pixel size: the volume's shadow exactly fills the detector,
  d_det = 2 DSD R / ((DSO - R) n_det) with R half the volume width.
* Angles theta_a = 2 pi a / A, a = 0..A-1 (uniform over 360 degrees).
* Phantoms: sums of ellipsoids, each adding its density at voxel centres that
  fall inside it (point-sampled, piecewise constant).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DSO_MM = 1000.0
DSD_MM = 1536.0


def detector_pixel(n_det: int, half_width_mm: float, dso: float = DSO_MM,
                   dsd: float = DSD_MM) -> float:
    """Pixel pitch at which the volume's shadow fills n_det pixels."""
    return 2.0 * dsd * half_width_mm / ((dso - half_width_mm) * n_det)


def geometry(n_voxel, d_voxel, n_det, d_det, *, dso=DSO_MM, dsd=DSD_MM,
             off_origin=(0.0, 0.0, 0.0), off_det=(0.0, 0.0), accuracy=0.5) -> dict:
    """Geometry descriptor with the C-ABI field names.

    n_voxel = (nx, ny, nz); d_voxel = (dx, dy, dz) mm; n_det = (nu, nv);
    d_det = (du, dv) mm; accuracy = ray step in voxels.
    """
    if np.isscalar(n_voxel):
        n_voxel = (int(n_voxel),) * 3
    if np.isscalar(d_voxel):
        d_voxel = (float(d_voxel),) * 3
    if np.isscalar(n_det):
        n_det = (int(n_det),) * 2
    if np.isscalar(d_det):
        d_det = (float(d_det),) * 2
    return {
        "DSO": float(dso),
        "DSD": float(dsd),
        "n_voxel": tuple(int(v) for v in n_voxel),
        "d_voxel": tuple(float(v) for v in d_voxel),
        "off_origin": tuple(float(v) for v in off_origin),
        "n_det": tuple(int(v) for v in n_det),
        "d_det": tuple(float(v) for v in d_det),
        "off_det": tuple(float(v) for v in off_det),
        "accuracy": float(accuracy),
    }


def angles(n: int, first: float = 0.0) -> np.ndarray:
    """Uniform angles over 360 degrees (float64 radians)."""
    return first + 2.0 * math.pi * np.arange(n, dtype=np.float64) / n


def cube_geometry(n: int, n_det: int, *, fov_mm: float = 256.0, d_voxel: float | None = None,
                  accuracy: float = 0.5) -> dict:
    """N^3 volume over a cubic field of view; detector sized to its shadow."""
    d = fov_mm / n if d_voxel is None else float(d_voxel)
    half = 0.5 * n * d
    return geometry(n, d, n_det, detector_pixel(n_det, half), accuracy=accuracy)


# Named workloads: (geometry, number of angles).
def workload(name: str):
    """Geometry and angles of a named workload.

    small_64     64^3, 1 mm voxels, 128^2 detector of 0.8 mm, 100 angles
    cgls_512     512^3, 0.5 mm voxels, 512^2 detector, 360 angles
    mixed_1024   1024^3, 0.25 mm voxels, 1024^2 detector, 720 angles
    ooc_3072     3072^3, 1/12 mm voxels, 3072^2 detector, 1500 angles
    """
    if name == "small_64":
        g = geometry(64, 1.0, 128, 0.8)
        return g, angles(100)
    if name == "cgls_512":
        return cube_geometry(512, 512), angles(360)
    if name == "mixed_1024":
        return cube_geometry(1024, 1024), angles(720)
    if name == "ooc_3072":
        return cube_geometry(3072, 3072), angles(1500)
    raise KeyError(name)


# ------------------------------------------------------------------ phantoms

@dataclass
class Ellipsoid:
    centre: tuple      # mm (x, y, z)
    axes: tuple        # semi-axes in mm
    rot: np.ndarray    # 3x3 rotation (rows = ellipsoid axes in world frame)
    density: float


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ellipsoids(n: int, d: float, count: int, seed: int,
                      r_vox=(5.0, 80.0)) -> list[Ellipsoid]:
    """Seeded random ellipsoids inside the sphere inscribed in an n^3 volume.

    Semi-axes U(r_vox) voxels (capped so each ellipsoid fits the inscribed
    sphere), centre uniform in the ball that keeps it inside, uniform random
    rotation, density U(0, 1).  r_vox is given for a 512^3 grid and scales with
    n / 512 so the phantom looks the same at every resolution.
    """
    rng = np.random.default_rng(seed)
    radius = 0.5 * n * d * 0.9
    scale = n / 512.0
    out = []
    for _ in range(count):
        axes = rng.uniform(r_vox[0], r_vox[1], size=3) * scale * d
        axes = np.minimum(axes, 0.45 * radius)
        rmax = float(axes.max())
        ball = max(radius - rmax, 0.0)
        while True:
            c = rng.uniform(-1.0, 1.0, size=3)
            if np.dot(c, c) <= 1.0:
                break
        out.append(Ellipsoid(tuple(c * ball), tuple(axes), _random_rotation(rng),
                             float(rng.uniform(0.0, 1.0))))
    return out


def nested_ellipsoids_10(n: int, d: float, seed: int = 1) -> list[Ellipsoid]:
    """Seeded 10-ellipsoid head-like stand-in (densities in [0, 1]).

    A large outer shell, a slightly smaller inner body cancelling most of it,
    and eight small inclusions, with random axes and orientations.  It takes
    the place of a published head phantom, which is not reproduced here.
    """
    rng = np.random.default_rng(seed)
    R = 0.5 * n * d
    ident = np.eye(3)
    out = [Ellipsoid((0.0, 0.0, 0.0), (0.69 * R, 0.92 * R, 0.81 * R), ident, 1.0),
           Ellipsoid((0.0, -0.018 * R, 0.0), (0.66 * R, 0.87 * R, 0.78 * R), ident, -0.8)]
    for _ in range(8):
        axes = rng.uniform(0.05, 0.3, size=3) * R
        c = rng.uniform(-0.4, 0.4, size=3) * R
        out.append(Ellipsoid(tuple(c), tuple(axes), _random_rotation(rng),
                             float(rng.uniform(0.05, 0.3))))
    return out


def voxelize(ells: list[Ellipsoid], n_voxel, d_voxel, off_origin=(0.0, 0.0, 0.0),
             dtype=np.float32, z_range=None) -> np.ndarray:
    """Sum of ellipsoid densities at voxel centres; array (nz, ny, nx).

    z_range=(z0, z1) voxelises only planes z0 <= k < z1 (for slab-wise
    generation of volumes larger than host memory budgets).
    """
    nx, ny, nz = n_voxel
    dx, dy, dz = d_voxel
    z0, z1 = (0, nz) if z_range is None else z_range
    vol = np.zeros((z1 - z0, ny, nx), dtype=np.float64)
    xs = (np.arange(nx) - 0.5 * (nx - 1)) * dx + off_origin[0]
    ys = (np.arange(ny) - 0.5 * (ny - 1)) * dy + off_origin[1]
    zs = (np.arange(z0, z1) - 0.5 * (nz - 1)) * dz + off_origin[2]
    for e in ells:
        r = max(e.axes)
        ix = np.nonzero(np.abs(xs - e.centre[0]) <= r)[0]
        iy = np.nonzero(np.abs(ys - e.centre[1]) <= r)[0]
        iz = np.nonzero(np.abs(zs - e.centre[2]) <= r)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        X = xs[ix][None, None, :] - e.centre[0]
        Y = ys[iy][None, :, None] - e.centre[1]
        Z = zs[iz][:, None, None] - e.centre[2]
        q = 0.0
        for a in range(3):
            comp = e.rot[0, a] * X + e.rot[1, a] * Y + e.rot[2, a] * Z
            q = q + (comp / e.axes[a]) ** 2
        inside = q <= 1.0
        sub = vol[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
        sub += np.where(inside, e.density, 0.0)
    return vol.astype(dtype)


def voxelize_torch(ells: list[Ellipsoid], n_voxel, d_voxel, z_range, device,
                   off_origin=(0.0, 0.0, 0.0)):
    """voxelize() for planes z_range[0] <= k < z_range[1], evaluated with torch
    in FP64 on `device` (for volumes whose numpy voxelisation would take too
    long); float32 tensor (z1 - z0, ny, nx).  Voxels exactly on an ellipsoid's
    surface may fall on the other side than in voxelize()."""
    import torch

    nx, ny, nz = n_voxel
    dx, dy, dz = d_voxel
    z0, z1 = z_range
    f64 = dict(dtype=torch.float64, device=device)
    xs = (torch.arange(nx, **f64) - 0.5 * (nx - 1)) * dx + off_origin[0]
    ys = (torch.arange(ny, **f64) - 0.5 * (ny - 1)) * dy + off_origin[1]
    zs = (torch.arange(z0, z1, **f64) - 0.5 * (nz - 1)) * dz + off_origin[2]
    vol = torch.zeros((z1 - z0, ny, nx), **f64)
    for e in ells:
        r = max(e.axes)
        ix = torch.nonzero((xs - e.centre[0]).abs() <= r).flatten()
        iy = torch.nonzero((ys - e.centre[1]).abs() <= r).flatten()
        iz = torch.nonzero((zs - e.centre[2]).abs() <= r).flatten()
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        xa, xb = int(ix[0]), int(ix[-1]) + 1
        ya, yb = int(iy[0]), int(iy[-1]) + 1
        za, zb = int(iz[0]), int(iz[-1]) + 1
        X = (xs[xa:xb] - e.centre[0])[None, None, :]
        Y = (ys[ya:yb] - e.centre[1])[None, :, None]
        Z = (zs[za:zb] - e.centre[2])[:, None, None]
        q = 0.0
        for a in range(3):
            comp = e.rot[0, a] * X + e.rot[1, a] * Y + e.rot[2, a] * Z
            q = q + (comp / e.axes[a]) ** 2
        vol[za:zb, ya:yb, xa:xb] += torch.where(q <= 1.0, e.density, 0.0)
    return vol.float()


def phantom(name: str, n: int, d: float, seed: int | None = None, dtype=np.float32,
            z_range=None) -> np.ndarray:
    """Named phantoms: 'head10' (10 nested ellipsoids) or 'ellipsoids50'."""
    if name == "head10":
        ells = nested_ellipsoids_10(n, d, 1 if seed is None else seed)
    elif name == "ellipsoids50":
        ells = random_ellipsoids(n, d, 50, 2 if seed is None else seed)
    else:
        raise KeyError(name)
    return voxelize(ells, (n, n, n), (d, d, d), dtype=dtype, z_range=z_range)


def add_noise(b: np.ndarray, sigma_rel: float, seed: int, object_only: bool = False) -> np.ndarray:
    """Gaussian noise with standard deviation sigma_rel * max(b), seeded.

    object_only=True adds it only to rays that cross the object (b > 0): rays
    that only graze the volume's support have a near-zero length, and noise
    there is amplified by SART's row weights 1/(A 1)."""
    rng = np.random.default_rng(seed)
    sigma = sigma_rel * float(np.max(b))
    noise = rng.normal(0.0, sigma, size=b.shape)
    if object_only:
        noise = np.where(b > 0, noise, 0.0)
    return (b + noise).astype(b.dtype)


def random_volume(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Uniform(0, 1) volume (nz, ny, nx), seeded."""
    return np.random.default_rng(seed).random(shape).astype(dtype)


def random_rays(n_angles: int, nv: int, nu: int, count: int, seed: int) -> np.ndarray:
    """Seeded (a, q, p) triplets, int64 array (count, 3)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n_angles, count), rng.integers(0, nv, count),
                     rng.integers(0, nu, count)], axis=1).astype(np.int64)


def random_voxels(nx: int, ny: int, nz: int, count: int, seed: int) -> np.ndarray:
    """Seeded (i, j, k) triplets, int64 array (count, 3)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, nx, count), rng.integers(0, ny, count),
                     rng.integers(0, nz, count)], axis=1).astype(np.int64)
