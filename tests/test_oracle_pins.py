"""Pins of the FP64 oracle against results fixed by the mathematics.

Every test here runs on the CPU and touches only ``oracle`` and the
independent computations in ``pins``; none uses the CUDA library.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_03748_gb300 import synth
from tests import pins


def tiny_geo(nx=10, ny=9, nz=8, nu=15, nv=11, d=(1.0, 1.1, 0.9), du=(1.3, 1.2),
             off_origin=(0.3, -0.2, 0.4), off_det=(0.7, -0.5), accuracy=0.5):
    """Anisotropic, offset, non-square geometry: index mix-ups show up here."""
    return synth.geometry((nx, ny, nz), d, (nu, nv), du, dso=60.0, dsd=95.0,
                          off_origin=off_origin, off_det=off_det, accuracy=accuracy)


# ------------------------------------------------------------ forward Ax

@pytest.mark.parametrize("n", [7, 8, 16])
def test_constant_volume_central_ray_is_exact(n):
    """A constant volume c and the central ray (odd detector, theta = 0 and
    90 deg): the interpolant ramps linearly over the outer half-voxels, so the
    line integral is c * n * d, and midpoint quadrature with the kinks on
    its grid reproduces it exactly."""
    c = 0.37
    geo = synth.geometry(n, 1.25, 9, 1.0, dso=50.0, dsd=80.0)
    vol = np.full((n, n, n), c)
    ang = np.array([0.0, math.pi / 2, math.pi])
    proj = oracle.forward(geo, ang, vol)
    for a in range(3):
        assert proj[a, 4, 4] == pytest.approx(c * n * 1.25, rel=1e-12)


def test_midpoint_converges_to_exact_integral_second_order():
    """Ax(h) -> the exact integral of the trilinear interpolant (computed by
    splitting at voxel planes + Gauss-Legendre), with error O(h^2)."""
    geo = tiny_geo()
    rng = np.random.default_rng(0)
    vol = rng.random((8, 9, 10))
    ang = np.array([0.3, 1.9, 4.0])
    rays = [(a, q, p) for a in range(3) for q in (1, 5, 9) for p in (2, 6, 7, 12)]
    exact = np.array([pins.exact_ray_integral(geo, vol, ang[a], p, q) for a, q, p in rays])
    assert np.count_nonzero(exact) > len(rays) // 2
    errs = []
    for acc in (0.2, 0.1, 0.05):
        g = dict(geo, accuracy=acc)
        approx = oracle.forward_rays(g, ang, vol, np.array(rays))
        errs.append(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    assert errs[0] < 2e-3
    for e0, e1 in zip(errs, errs[1:]):
        assert 2.5 < e0 / e1 < 6.0, errs
    fine = oracle.forward_rays(dict(geo, accuracy=0.002), ang, vol, np.array(rays))
    assert np.linalg.norm(fine - exact) / np.linalg.norm(exact) < 1e-5


def test_brute_force_fine_sampling_8cubed():
    """8^3 volume, every ray of two angles: oracle at 1e-3 voxel steps equals
    the exact integral of the interpolant."""
    geo = synth.geometry(8, 1.0, (12, 10), 1.1, dso=40.0, dsd=70.0, accuracy=0.001)
    vol = np.random.default_rng(3).random((8, 8, 8))
    ang = np.array([0.4, 2.2])
    proj = oracle.forward(geo, ang, vol)
    exact = np.array([[[pins.exact_ray_integral(geo, vol, ang[a], p, q) for p in range(12)]
                       for q in range(10)] for a in range(2)])
    assert np.abs(proj - exact).max() <= 1e-6 * np.abs(exact).max()


def test_rotation_by_90_degrees_is_a_transpose():
    """Projecting at theta + 90 deg the volume rotated by +90 deg about z
    equals projecting the original at theta."""
    n = 12
    geo = synth.geometry((n, n, 7), (0.8, 0.8, 1.1), (17, 9), (1.0, 1.2), dso=45.0, dsd=70.0,
                         off_det=(0.3, 0.2))
    vol = np.random.default_rng(1).random((7, n, n))
    rot = vol[:, ::-1, :].transpose(0, 2, 1)
    th = np.array([0.25, 1.0, 2.5])
    a = oracle.forward(geo, th, vol)
    b = oracle.forward(geo, th + math.pi / 2, rot)
    np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("theta", [0.0, math.pi / 2, 0.9, 3.7])
def test_single_voxel_lands_where_the_frame_says(theta):
    """A lone voxel projects around the detector point that the
    source->voxel line meets: the centroid of its footprint, sampled by
    pixels 8x finer than the footprint, sits within 0.02 px of it (perspective
    and pixel sampling move it by less than 0.01 px here)."""
    geo = tiny_geo(nx=16, ny=16, nz=12, nu=161, nv=121, d=(1.0, 1.0, 1.0), du=(0.225, 0.225))
    vol = np.zeros((12, 16, 16))
    i, j, k = 11, 4, 8
    vol[k, j, i] = 1.0
    proj = oracle.forward(dict(geo, accuracy=0.05), np.array([theta]), vol)[0]
    q_idx, p_idx = np.mgrid[0:121, 0:161]
    m = proj.sum()
    pc, qc = (proj * p_idx).sum() / m, (proj * q_idx).sum() / m
    p, q, _ = pins.detector_hit(geo, theta, pins.voxel_centre(geo, i, j, k))
    assert abs(pc - p) < 0.02 and abs(qc - q) < 0.02
    # a mirrored frame (e_u flipped) would put it 2|p - centre| px away
    assert abs(p - 80.0 - geo["off_det"][0] / 0.225) > 2.0


def test_voxelised_ellipsoids_converge_to_analytic_chords():
    """Ax of the point-sampled phantom approaches sum(density x chord) as the
    grid refines (same phantom in mm)."""
    fov = 64.0
    rng = np.random.default_rng(7)
    ells = []
    for _ in range(3):
        ells.append(synth.Ellipsoid(tuple(rng.uniform(-8, 8, 3)), tuple(rng.uniform(6, 14, 3)),
                                    synth._random_rotation(rng), float(rng.uniform(0.2, 1.0))))
    ang = np.array([0.2, 1.3, 2.9])
    errs = []
    for n in (16, 32, 64):
        d = fov / n
        geo = synth.geometry(n, d, (24, 20), 3.0, dso=200.0, dsd=300.0)
        vol = synth.voxelize(ells, (n, n, n), (d, d, d), dtype=np.float64)
        proj = oracle.forward(geo, ang, vol)
        ref = np.zeros_like(proj)
        for a, th in enumerate(ang):
            S = pins.frame(geo, th)[0]
            for q in range(20):
                for p in range(24):
                    P = pins.pixel_centre(geo, th, p, q)
                    ref[a, q, p] = sum(e.density * pins.ellipsoid_chord(S, P, e.centre, e.axes,
                                                                        e.rot) for e in ells)
        errs.append(np.linalg.norm(proj - ref) / np.linalg.norm(ref))
    # boundary voxelisation error shrinks about linearly with the voxel size
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 2.5 and errs[2] < 0.05, errs


# -------------------------------------------------------- exact adjoint

def test_exact_adjoint_dot_product():
    """<A x, y> = <x, A^T y> to rounding."""
    geo = tiny_geo()
    rng = np.random.default_rng(11)
    ang = np.array([0.1, 0.9, 2.0, 3.3, 5.5])
    x = rng.random((8, 9, 10))
    y = rng.random((5, 11, 15))
    lhs = np.sum(oracle.forward(geo, ang, x) * y)
    rhs = np.sum(x * oracle.adjoint(geo, ang, y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_exact_adjoint_equals_dense_transpose():
    """A^T y equals the transpose of the matrix built column by column from
    Ax applied to unit vectors."""
    geo = tiny_geo(nx=4, ny=3, nz=3, nu=6, nv=5)
    ang = np.array([0.2, 1.7, 4.1])
    N = 4 * 3 * 3
    A = np.stack([oracle.forward(geo, ang, np.eye(N)[c].reshape(3, 3, 4)).ravel()
                  for c in range(N)], axis=1)
    y = np.random.default_rng(2).random(A.shape[0])
    np.testing.assert_allclose(oracle.adjoint(geo, ang, y.reshape(3, 5, 6)).ravel(), A.T @ y,
                               rtol=1e-12, atol=1e-14)


def test_adjoint_at_selected_voxels_matches_full_scatter():
    geo = tiny_geo()
    ang = np.array([0.1, 2.0, 4.4])
    y = np.random.default_rng(5).random((3, 11, 15))
    full = oracle.adjoint(geo, ang, y)
    vox = synth.random_voxels(10, 9, 8, 40, seed=9)
    sel = oracle.adjoint_voxels(geo, ang, y, vox)
    np.testing.assert_allclose(sel, full[vox[:, 2], vox[:, 1], vox[:, 0]], rtol=1e-12,
                               atol=1e-14)


# ------------------------------------------------------ backprojection

@pytest.mark.parametrize("theta", [0.0, 0.7, 2.9])
def test_fdk_backprojection_of_one_pixel(theta):
    """Backprojecting an image that is 1 at pixel (p0, q0): each voxel gets
    w_FDK * tent(p - p0) * tent(q - q0), with (p, q) the detector hit of the
    source->voxel line (plane intersection) and w = (DSO/depth)^2."""
    geo = tiny_geo(nx=12, ny=12, nz=10, nu=21, nv=17, du=(0.8, 0.8))
    img = np.zeros((1, 17, 21))
    p0, q0 = 10, 9
    img[0, q0, p0] = 1.0
    bp = oracle.backward(geo, np.array([theta]), img, oracle.BP_FDK)
    ref = np.zeros_like(bp)
    for k in range(10):
        for j in range(12):
            for i in range(12):
                p, q, depth = pins.detector_hit(geo, theta, pins.voxel_centre(geo, i, j, k))
                tent = max(0.0, 1 - abs(p - p0)) * max(0.0, 1 - abs(q - q0))
                ref[k, j, i] = (geo["DSO"] / depth) ** 2 * tent
    assert np.count_nonzero(ref) > 10
    np.testing.assert_allclose(bp, ref, rtol=1e-10, atol=1e-13)


def test_fdk_backprojection_of_ones_at_isocentre():
    """The isocentre voxel projects to the detector centre with weight 1 at
    every angle, so backprojecting ones gives the number of angles."""
    geo = synth.geometry(9, 1.0, 15, 1.0, dso=50.0, dsd=80.0)
    ang = synth.angles(13)
    bp = oracle.backward(geo, ang, np.ones((13, 15, 15)), oracle.BP_FDK)
    assert bp[4, 4, 4] == pytest.approx(13.0, rel=1e-13)


def test_matched_backprojection_approximates_exact_adjoint():
    """The pseudo-matched weights make the voxel-driven BP approximate the
    transpose of the ray-driven projector: on smooth data the two agree to a
    few percent inside the field of view (the weights' derivation: voxel
    volume over the ray tube's cross-section at the voxel)."""
    n = 24
    geo = synth.geometry(n, 1.0, 48, 0.75, dso=100.0, dsd=150.0)
    ang = synth.angles(24)
    q_idx, p_idx = np.mgrid[0:48, 0:48]
    y = np.stack([1.0 + 0.3 * np.sin(0.07 * p_idx + 0.05 * q_idx + a) for a in range(24)])
    m = oracle.backward(geo, ang, y, oracle.BP_MATCHED)
    e = oracle.adjoint(geo, ang, y)
    core = (slice(4, n - 4),) * 3
    rel = np.linalg.norm(m[core] - e[core]) / np.linalg.norm(e[core])
    assert rel < 0.03, rel
    # the FDK-weighted BP is a different operator (no voxel-volume factor)
    f = oracle.backward(geo, ang, y, oracle.BP_FDK)
    assert np.linalg.norm(f[core] - e[core]) / np.linalg.norm(e[core]) > 0.2


def test_backprojection_at_selected_voxels_matches_full():
    geo = tiny_geo()
    ang = np.array([0.3, 1.1, 5.0])
    y = np.random.default_rng(4).random((3, 11, 15))
    vox = synth.random_voxels(10, 9, 8, 30, seed=1)
    for mode in (oracle.BP_MATCHED, oracle.BP_FDK):
        full = oracle.backward(geo, ang, y, mode)
        sel = oracle.backward_voxels(geo, ang, y, vox, mode)
        np.testing.assert_allclose(sel, full[vox[:, 2], vox[:, 1], vox[:, 0]], rtol=1e-14)


def test_forward_at_selected_rays_matches_full():
    geo = tiny_geo()
    ang = np.array([0.3, 1.1, 5.0])
    vol = np.random.default_rng(4).random((8, 9, 10))
    full = oracle.forward(geo, ang, vol)
    rays = synth.random_rays(3, 11, 15, 50, seed=2)
    np.testing.assert_allclose(oracle.forward_rays(geo, ang, vol, rays),
                               full[rays[:, 0], rays[:, 1], rays[:, 2]], rtol=1e-14)


# ------------------------------------------------------------------ TV

def tv_numpy(f, eps):
    """TV_eps by array differencing (independent of the oracle's loops)."""
    dx = np.diff(f, axis=2, prepend=f[:, :, :1])
    dy = np.diff(f, axis=1, prepend=f[:, :1, :])
    dz = np.diff(f, axis=0, prepend=f[:1, :, :])
    return float(np.sum(np.sqrt(dx * dx + dy * dy + dz * dz + eps)))


def test_tv_value_matches_array_differencing():
    f = np.random.default_rng(0).random((5, 6, 7))
    assert oracle.tv_value(f, 1e-3) == pytest.approx(tv_numpy(f, 1e-3), rel=1e-13)


def test_tv_gradient_matches_central_differences():
    f = np.random.default_rng(1).random((5, 6, 7))
    eps = 1e-2
    g = oracle.tv_grad(f, eps)
    h = 1e-6
    fd = np.empty_like(f)
    for idx in np.ndindex(f.shape):
        fp = f.copy()
        fm = f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd[idx] = (tv_numpy(fp, eps) - tv_numpy(fm, eps)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_tv_gradient_zero_on_constant_and_steps_decrease_tv():
    c = np.full((4, 5, 6), 0.3)
    assert np.abs(oracle.tv_grad(c, 1e-8)).max() == 0.0
    assert np.array_equal(oracle.tv_steps(c, 3, 0.1, 1e-8), c)
    f = np.random.default_rng(2).random((6, 6, 6))
    tv0 = oracle.tv_value(f, 1e-8)
    f1 = oracle.tv_steps(f, 5, 0.05, 1e-8)
    assert oracle.tv_value(f1, 1e-8) < tv0


def test_tv_gradient_at_selected_voxels():
    f = np.random.default_rng(3).random((6, 7, 8))
    g = oracle.tv_grad(f, 1e-4)
    vox = synth.random_voxels(8, 7, 6, 25, seed=3)
    np.testing.assert_allclose(oracle.tv_grad_voxels(f, 1e-4, vox),
                               g[vox[:, 2], vox[:, 1], vox[:, 0]], rtol=1e-14)


# -------------------------------------------------------------- solvers

def dense_operators(geo, ang):
    nx, ny, nz = geo["n_voxel"]
    nu, nv = geo["n_det"]
    N, M = nx * ny * nz, len(ang) * nu * nv
    A = np.stack([oracle.forward(geo, ang, np.eye(N)[c].reshape(nz, ny, nx)).ravel()
                  for c in range(N)], axis=1)
    Bm = np.stack([oracle.backward(geo, ang, np.eye(M)[c].reshape(len(ang), nv, nu)).ravel()
                   for c in range(M)], axis=1)
    return A, Bm


def test_sirt_equals_dense_iteration():
    geo = tiny_geo(nx=4, ny=4, nz=3, nu=6, nv=5)
    ang = synth.angles(5)
    A, Bm = dense_operators(geo, ang)
    b = A @ np.random.default_rng(0).random(A.shape[1])
    row, col = A @ np.ones(A.shape[1]), Bm @ np.ones(A.shape[0])
    assert np.any(row == 0.0)           # some rays miss: the zero guard matters
    W = np.where(row > 1e-12, 1.0 / np.where(row > 1e-12, row, 1.0), 0.0)
    V = np.where(col > 1e-12, 1.0 / np.where(col > 1e-12, col, 1.0), 0.0)
    x = np.zeros(A.shape[1])
    for _ in range(6):
        x = x + V * (Bm @ (W * (b - A @ x)))
    xo, res = oracle.sirt(geo, ang, b.reshape(5, 5, 6), 6)
    np.testing.assert_allclose(xo.ravel(), x, rtol=1e-11, atol=1e-13)
    assert np.all(np.diff(res) < 0)


def test_os_sart_with_one_subset_is_sirt():
    geo = tiny_geo(nx=5, ny=4, nz=3, nu=7, nv=5)
    ang = synth.angles(6)
    vol = np.random.default_rng(1).random((3, 4, 5))
    b = oracle.forward(geo, ang, vol)
    x1, r1 = oracle.sirt(geo, ang, b, 4)
    x2, r2 = oracle.os_sart(geo, ang, b, 4, subset=6)
    np.testing.assert_allclose(x2, x1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(r2, r1, rtol=1e-13)


def test_os_sart_subsets_reduce_error_on_noiseless_data():
    geo = synth.geometry(12, 1.0, 20, 1.0, dso=60.0, dsd=90.0)
    ang = synth.angles(20)
    truth = synth.voxelize(synth.random_ellipsoids(12, 1.0, 4, seed=5, r_vox=(100, 200)),
                           (12, 12, 12), (1.0, 1.0, 1.0), dtype=np.float64)
    b = oracle.forward(geo, ang, truth)
    errs = []
    for it in (1, 3, 6):
        x, _ = oracle.os_sart(geo, ang, b, it, subset=5)
        errs.append(np.linalg.norm(x - truth))
    assert errs[0] > errs[1] > errs[2]


def test_cgls_with_exact_adjoint_reaches_least_squares():
    """With the exact transpose, CGLS is CG on the normal equations: the
    residual norm decreases monotonically and it reaches lstsq."""
    geo = tiny_geo(nx=3, ny=3, nz=2, nu=6, nv=4)
    ang = synth.angles(4)
    A, _ = dense_operators(geo, ang)
    rng = np.random.default_rng(6)
    b = A @ rng.random(A.shape[1]) + 0.01 * rng.standard_normal(A.shape[0])
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    x, res = oracle.cgls(geo, ang, b.reshape(4, 4, 6), 40, bp="adjoint")
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    np.testing.assert_allclose(x.ravel(), x_ls, rtol=1e-6, atol=1e-8)
    # textbook CG on A^T A x = A^T b from zero: same first iterates
    xc = np.zeros(A.shape[1])
    r = A.T @ b
    pdir = r.copy()
    for _ in range(3):
        Ap = A.T @ (A @ pdir)
        al = (r @ r) / (pdir @ Ap)
        xc = xc + al * pdir
        rn = r - al * Ap
        pdir = rn + (rn @ rn) / (r @ r) * pdir
        r = rn
    x3, _ = oracle.cgls(geo, ang, b.reshape(4, 4, 6), 3, bp="adjoint")
    np.testing.assert_allclose(x3.ravel(), xc, rtol=1e-9, atol=1e-12)


# ------------------------------------------------- Siddon (ray-voxel) projector

def all_rays(geo, ang):
    nu, nv = geo["n_det"]
    return [(a, q, p) for a in range(len(ang)) for q in range(nv) for p in range(nu)]


def test_siddon_constant_volume_gives_box_chord():
    """Constant c: c times the chord of the segment through the volume's box."""
    geo = tiny_geo()
    ang = np.array([0.0, 0.7, 1.5707963267948966, 2.6, 4.0])
    c = 0.83
    got = oracle.siddon_forward(geo, ang, np.full((8, 9, 10), c))
    lo, hi = pins.volume_box(geo)
    want = np.array([c * pins.box_chord(pins.frame(geo, ang[a])[0],
                                        pins.pixel_centre(geo, ang[a], p, q), lo, hi)
                     for a, q, p in all_rays(geo, ang)]).reshape(got.shape)
    assert want.max() > 5.0
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("ijk", [(0, 0, 0), (9, 8, 7), (4, 5, 3), (7, 1, 6)])
def test_siddon_single_voxel_is_its_box_chord(ijk):
    """One voxel of value 1: every ray gets its intersection length with that
    voxel's box (corner voxels included)."""
    geo = tiny_geo()
    ang = np.array([0.3, 2.2, 5.1])
    vol = np.zeros((8, 9, 10))
    vol[ijk[2], ijk[1], ijk[0]] = 1.0
    got = oracle.siddon_forward(geo, ang, vol)
    lo, hi = pins.voxel_box(geo, *ijk)
    want = np.array([pins.box_chord(pins.frame(geo, ang[a])[0],
                                    pins.pixel_centre(geo, ang[a], p, q), lo, hi)
                     for a, q, p in all_rays(geo, ang)]).reshape(got.shape)
    assert want.max() > 0.5
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_siddon_brute_force_fine_sampling():
    """The midpoint rule on the piecewise-constant volume converges to the
    Siddon value (first order in the step: the integrand jumps at voxel
    faces)."""
    geo = tiny_geo(nx=6, ny=5, nz=4, nu=7, nv=5)
    ang = np.array([0.4, 2.9])
    vol = np.random.default_rng(5).random((4, 5, 6))
    rays = [(0, 2, 3), (1, 1, 5), (0, 4, 0), (1, 3, 2)]
    sid = oracle.siddon_forward_rays(geo, ang, vol, np.array(rays))
    lo_b, hi_b = pins.volume_box(geo)
    for (a, q, p), s in zip(rays, sid):
        S = pins.frame(geo, ang[a])[0]
        P = pins.pixel_centre(geo, ang[a], p, q)
        errs = []
        for m in (2000, 20000):
            t = (np.arange(m) + 0.5) / m
            X = S[None, :] + t[:, None] * (P - S)[None, :]
            idx = np.floor(pins.world_to_index(geo, X) + 0.5).astype(np.int64)
            n = np.array(geo["n_voxel"])
            ok = np.all((idx >= 0) & (idx < n), axis=1)
            vals = np.zeros(m)
            vals[ok] = vol[idx[ok, 2], idx[ok, 1], idx[ok, 0]]
            errs.append(abs(vals.sum() * np.linalg.norm(P - S) / m - s))
        assert errs[1] < 0.3 * errs[0] + 1e-9 and errs[1] < 2e-2 * max(abs(s), 1e-9) + 1e-6


def test_siddon_adjoint_dot_product_and_dense_transpose():
    geo = tiny_geo()
    rng = np.random.default_rng(12)
    ang = np.array([0.1, 1.9, 3.7])
    x = rng.random((8, 9, 10))
    y = rng.random((3, 11, 15))
    lhs = np.sum(oracle.siddon_forward(geo, ang, x) * y)
    rhs = np.sum(x * oracle.siddon_adjoint(geo, ang, y))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    small = tiny_geo(nx=3, ny=3, nz=2, nu=5, nv=4)
    a2 = np.array([0.5, 2.5])
    N = 18
    A = np.stack([oracle.siddon_forward(small, a2, np.eye(N)[c].reshape(2, 3, 3)).ravel()
                  for c in range(N)], axis=1)
    yy = rng.random(A.shape[0])
    np.testing.assert_allclose(oracle.siddon_adjoint(small, a2, yy.reshape(2, 4, 5)).ravel(),
                               A.T @ yy, rtol=1e-12, atol=1e-14)


def test_siddon_and_interpolated_projectors_agree_on_smooth_volumes():
    """Both projectors integrate the same smooth object along the same rays
    (the two give nearly the same reconstructions, Sec. 3.1): on a sampled
    Gaussian blob their difference shrinks as the grid is refined, and the
    total ray sums agree (both conserve the object's mass)."""
    rels = []
    for n in (32, 64):
        geo = synth.geometry(n, 32.0 / n, 48, 1.0, dso=200.0, dsd=300.0)
        ang = synth.angles(8)
        c = (np.arange(n) - (n - 1) / 2.0) * 32.0 / n
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        vol = np.exp(-(x ** 2 + (1.3 * y) ** 2 + (0.8 * z) ** 2) / (2 * 6.0 ** 2))
        a = oracle.siddon_forward(geo, ang, vol)
        b = oracle.forward(geo, ang, vol)
        rels.append(np.linalg.norm(a - b) / np.linalg.norm(b))
        assert a.sum() == pytest.approx(b.sum(), rel=1e-3)
    assert rels[1] < 0.5 * rels[0] and rels[1] < 1e-2


def test_siddon_cgls_with_exact_adjoint_reaches_least_squares():
    """CGLS on the Siddon projector with its transpose reaches lstsq of the
    dense Siddon matrix (built from unit vectors; a detector and angle set
    for which that matrix has full column rank)."""
    geo = tiny_geo(nx=3, ny=3, nz=2, nu=8, nv=6)
    ang = synth.angles(6)
    N = 18
    A = np.stack([oracle.siddon_forward(geo, ang, np.eye(N)[c].reshape(2, 3, 3)).ravel()
                  for c in range(N)], axis=1)
    rng = np.random.default_rng(8)
    b = A @ rng.random(N) + 0.01 * rng.standard_normal(A.shape[0])
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.matrix_rank(A) == N
    x, res = oracle.cgls(geo, ang, b.reshape(6, 6, 8), 40, bp="adjoint", projector="siddon")
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    np.testing.assert_allclose(x.ravel(), x_ls, rtol=1e-6, atol=1e-8)


# ------------------------------------------------------------------- FDK

def test_ramp_kernel_is_the_band_limited_ramp():
    """The Ram-Lak coefficients are the Fourier series of |w| on the Nyquist
    band: sum_k h[k] exp(-2 pi i w k) = |w| for |w| <= 1/2 (unit spacing),
    up to the tail of the truncated series."""
    M = 200000
    h = oracle.ramp_kernel(M + 1)
    k = np.arange(-M, M + 1)
    for w in (0.0, 0.03, 0.11, 0.25, 0.37, 0.49):
        H = np.sum(h * np.cos(2 * np.pi * w * k))
        assert abs(H - abs(w)) < 1e-5, w


def test_fdk_angle_weights():
    np.testing.assert_allclose(oracle.fdk_angle_weights(synth.angles(7)), 2 * np.pi / 7,
                               rtol=1e-12)
    ang = np.random.default_rng(3).uniform(0, 2 * np.pi, 11)
    w = oracle.fdk_angle_weights(ang)
    assert w.sum() == pytest.approx(2 * np.pi, rel=1e-12)
    assert np.all(w > 0)


def test_fdk_reconstructs_a_uniform_ball():
    """Near-parallel cone (DSO 2 m, 48 mm ball of radius 15 voxels): FDK of
    the ball's projections returns its density inside and zero outside."""
    N = 48
    geo = synth.geometry(N, 1.0, 96, 1.0, dso=2000.0, dsd=3000.0)
    ang = synth.angles(180)
    c = np.arange(N) - (N - 1) / 2.0
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = x ** 2 + y ** 2 + z ** 2
    vol = (r2 <= 15.0 ** 2) * 0.7
    rec = oracle.fdk(geo, ang, oracle.forward(geo, ang, vol))
    inner, outer = r2 <= 11.0 ** 2, r2 >= 19.0 ** 2
    assert abs(rec[inner].mean() - 0.7) < 3e-3
    assert rec[inner].std() < 1e-2
    assert abs(rec[outer].mean()) < 3e-3


def test_fdk_wide_fan_mid_plane_is_exact_fan_beam():
    """In the mid-plane FDK is fan-beam FBP, exact up to discretisation.  An
    off-centre ball seen at fan angles up to ~20 degrees comes back at its
    density; dropping the cosine pre-weight would bias it by ~1 %."""
    N = 48
    geo = synth.geometry(N, 1.0, (256, 64), 1.0, dso=60.0, dsd=90.0)
    ang = synth.angles(360)
    c = np.arange(N) - (N - 1) / 2.0
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    vol = ((x - 13) ** 2 + y ** 2 + z ** 2 <= 7.0 ** 2) * 0.7
    rec = oracle.fdk(geo, ang, oracle.forward(geo, ang, vol))
    core = (np.abs(z) <= 0.5) & ((x - 13) ** 2 + y ** 2 <= 4 ** 2)
    assert abs(rec[core].mean() - 0.7) < 2.5e-3


# --------------------------------------------------------------- ROF TV

def test_rof_divergence_is_minus_gradient_transpose():
    rng = np.random.default_rng(14)
    u = rng.random((4, 5, 6))
    p = [rng.random((4, 5, 6)) for _ in range(3)]
    lhs = sum(np.sum(a * b) for a, b in zip(oracle.rof_grad(u), p))
    assert lhs == pytest.approx(-np.sum(u * oracle.rof_div(*p)), rel=1e-12)
    # one-voxel axes have no differences at all
    flat = rng.random((1, 5, 6))
    assert not oracle.rof_grad(flat)[2].any()


def test_rof_leaves_constants_and_solves_a_step_exactly():
    """A constant image is its own ROF solution; a two-level step (0 on a
    voxels, h on b voxels, constant across y and z) has the closed-form
    solution 1/(lam a) and h - 1/(lam b) (each level moves by the jump's
    unit TV weight over its mass)."""
    c = np.full((3, 4, 5), 0.42)
    np.testing.assert_allclose(oracle.rof_denoise(c, 0.7, 50), c, rtol=0, atol=1e-15)
    f = np.zeros((2, 3, 16))
    f[:, :, 6:] = 1.0
    lam = 1.0
    u = oracle.rof_denoise(f, lam, 1500)
    np.testing.assert_allclose(u[:, :, :6], 1.0 / (lam * 6), atol=1e-10)
    np.testing.assert_allclose(u[:, :, 6:], 1.0 - 1.0 / (lam * 10), atol=1e-10)


def test_rof_converged_point_is_a_minimum():
    """After many iterations on a random image, small perturbations in random
    directions do not lower the ROF objective."""
    rng = np.random.default_rng(15)
    f = rng.random((5, 6, 7))
    lam = 4.0
    u = oracle.rof_denoise(f, lam, 4000)
    J = oracle.rof_objective(u, f, lam)
    assert J < oracle.rof_objective(f, f, lam)
    for _ in range(20):
        d = rng.standard_normal(f.shape)
        assert oracle.rof_objective(u + 1e-3 * d, f, lam) >= J - 1e-9


# ------------------------------------------------ split TV (halo buffers)

def test_split_tv_with_one_slab_is_the_global_descent():
    f = np.random.default_rng(18).random((9, 7, 8))
    np.testing.assert_allclose(oracle.tv_steps_split(f, 5, 0.02, 1e-8, slab=9, depth=2),
                               oracle.tv_steps(f, 5, 0.02, 1e-8), rtol=1e-12, atol=1e-14)


def test_split_tv_single_step_moves_each_slab_along_the_exact_gradient():
    """One step: inside each slab the update is the exact gradient there
    (the one-plane buffer covers the stencil), scaled to length
    alpha sqrt(N_slab / N) (the uniform-distribution norm approximation)."""
    f = np.random.default_rng(19).random((10, 6, 7))
    alpha = 0.05
    out = oracle.tv_steps_split(f, 1, alpha, 1e-8, slab=3, depth=1)
    g = oracle.tv_grad(f, 1e-8)
    N = f.size
    for z0 in range(0, 10, 3):
        z1 = min(10, z0 + 3)
        gi = g[z0:z1]
        want = f[z0:z1] - alpha * np.sqrt(gi.size / N) * gi / np.linalg.norm(gi)
        np.testing.assert_allclose(out[z0:z1], want, rtol=1e-12, atol=1e-14)


def test_split_tv_buffer_as_deep_as_the_steps_is_enough():
    """k independent steps need a k-plane buffer: a deeper buffer (the whole
    volume) gives the same slab interiors; a shallower one does not."""
    f = np.random.default_rng(20).random((12, 5, 6))
    a = oracle.tv_steps_split(f, 3, 0.03, 1e-8, slab=4, depth=3)
    b = oracle.tv_steps_split(f, 3, 0.03, 1e-8, slab=4, depth=3, halo=12)
    c = oracle.tv_steps_split(f, 3, 0.03, 1e-8, slab=4, depth=3, halo=1)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
    assert np.abs(a - c).max() > 1e-6


# ------------------------------------------ OS-SART subsets and TV coupling

def dense_os_sart(A, Bm, b, na, subset, n_iter, order=None, global_v=False):
    """OS-SART written on dense matrices: rows of A and columns of Bm are
    angle-major, a subset is `subset` consecutive angles, W_s = 1/(A_s 1) and
    V_s = 1/(Bm_s 1) with the zero guard, subsets visited in `order`."""
    m = A.shape[0] // na
    blocks = [np.arange(s, min(s + subset, na)) for s in range(0, na, subset)]
    rows = [np.concatenate([np.arange(a * m, (a + 1) * m) for a in blk]) for blk in blocks]

    def recip(v):
        return np.where(v > 1e-12, 1.0 / np.where(v > 1e-12, v, 1.0), 0.0)

    V_all = recip(Bm @ np.ones(A.shape[0]))
    x = np.zeros(A.shape[1])
    res = []
    for _ in range(n_iter):
        rr = 0.0
        for s in (order if order is not None else range(len(blocks))):
            As, Bs = A[rows[s]], Bm[:, rows[s]]
            W = recip(As @ np.ones(A.shape[1]))
            V = V_all if global_v else recip(Bs @ np.ones(len(rows[s])))
            r = b[rows[s]] - As @ x
            rr += float(r @ r)
            x = x + V * (Bs @ (W * r))
        res.append(np.sqrt(rr))
    return x, np.array(res)


@pytest.mark.parametrize("subset", [2, 4])
def test_os_sart_subsets_equal_the_dense_per_subset_iteration(subset):
    """Sec. 3.2's OS-SART with 3 subsets of 2 angles and with a ragged split
    (4 + 2): the oracle equals the dense iteration with per-subset weights
    W_s, V_s and the subsets in acquisition order.  A global V, or the
    subsets visited in reverse, lands far away, so either mistake fails."""
    geo = tiny_geo(nx=4, ny=4, nz=3, nu=6, nv=5)
    ang = synth.angles(6)
    A, Bm = dense_operators(geo, ang)
    b = A @ np.random.default_rng(2).random(A.shape[1])
    x_ref, r_ref = dense_os_sart(A, Bm, b, 6, subset, 3)
    xo, ro = oracle.os_sart(geo, ang, b.reshape(6, 5, 6), 3, subset=subset)
    np.testing.assert_allclose(xo.ravel(), x_ref, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(ro, r_ref, rtol=1e-11)
    nb = (6 + subset - 1) // subset
    for wrong in (dense_os_sart(A, Bm, b, 6, subset, 3, global_v=True)[0],
                  dense_os_sart(A, Bm, b, 6, subset, 3, order=range(nb - 1, -1, -1))[0]):
        assert np.linalg.norm(wrong - x_ref) > 1e-3 * np.linalg.norm(x_ref)


def tv_grad_autograd(x: np.ndarray, eps: float) -> np.ndarray:
    """Gradient of TV_eps(f) = sum sqrt(Dx^2 + Dy^2 + Dz^2 + eps), backward
    differences with zero across the low boundary, by reverse-mode automatic
    differentiation of that sum (FP64, CPU) -- not the oracle's stencil."""
    import torch
    f = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    dz = torch.cat([torch.zeros_like(f[:1]), f[1:] - f[:-1]], 0)
    dy = torch.cat([torch.zeros_like(f[:, :1]), f[:, 1:] - f[:, :-1]], 1)
    dx = torch.cat([torch.zeros_like(f[:, :, :1]), f[:, :, 1:] - f[:, :, :-1]], 2)
    torch.sqrt(dx * dx + dy * dy + dz * dz + eps).sum().backward()
    return f.grad.numpy()


@pytest.mark.parametrize("n_iter", [1, 2])
def test_os_sart_tv_runs_after_each_full_sweep_with_the_update_norm_as_step(n_iter):
    """Sec. 2.3 couples the regulariser to the data step through the norm of
    the image update.  Each OS-SART+TV iteration here is the dense data
    sweep over all subsets, then tv_steps steps x <- x - a g/||g|| with
    a = tv_alpha * ||x_after_sweep - x_before_sweep|| and g from automatic
    differentiation of TV_eps.  TV before the sweep, after every subset, or
    a step scaled by ||x|| instead of the update would not match."""
    geo = tiny_geo(nx=4, ny=4, nz=3, nu=6, nv=5)
    ang = synth.angles(6)
    A, Bm = dense_operators(geo, ang)
    b = A @ np.random.default_rng(3).random(A.shape[1])
    tv_alpha, n_tv, eps = 0.3, 4, 1e-6
    x = np.zeros(A.shape[1])
    for _ in range(n_iter):
        x_prev = x.copy()
        # one full sweep from x: dense OS-SART iteration started there
        m = A.shape[0] // 6
        for s in range(3):
            rows = np.arange(2 * s * m, (2 * s + 2) * m)
            As, Bs = A[rows], Bm[:, rows]
            W = 1.0 / np.where(As.sum(1) > 1e-12, As.sum(1), np.inf)
            cs = Bs.sum(1)
            V = np.where(cs > 1e-12, 1.0 / np.where(cs > 1e-12, cs, 1.0), 0.0)
            x = x + V * (Bs @ (W * (b[rows] - As @ x)))
        a = tv_alpha * np.linalg.norm(x - x_prev)
        v = x.reshape(3, 4, 4)
        for _ in range(n_tv):
            g = tv_grad_autograd(v, eps)
            v = v - a * g / np.linalg.norm(g)
        x = v.ravel()
    xo, _ = oracle.os_sart(geo, ang, b.reshape(6, 5, 6), n_iter, subset=2, tv_steps_n=n_tv,
                           tv_alpha=tv_alpha, tv_eps=eps)
    np.testing.assert_allclose(xo.ravel(), x, rtol=1e-9, atol=1e-11)
    x_plain, _ = oracle.os_sart(geo, ang, b.reshape(6, 5, 6), n_iter, subset=2)
    assert np.linalg.norm(x_plain.ravel() - x) > 1e-3 * np.linalg.norm(x)  # TV mattered


def test_sample_count_is_the_chord_rule_on_the_enlarged_box():
    """The work count of Ax: per ray K = max(1, ceil(len/D - 1e-9)) with len
    the chord (mm) of the ray through the interpolant's support -- the box
    of voxel centres -1 .. n on each axis -- and D = accuracy * min(d); rays
    that miss it count 0.  The chord comes from world-space slab clipping
    of the rotated frame; summed over every ray it equals sample_count, and
    ray by ray the K the oracle places."""
    geo = tiny_geo(nx=9, ny=7, nz=5, nu=19, nv=13, d=(1.0, 1.2, 0.8), du=(1.1, 0.9),
                   off_origin=(0.37, -0.21, 0.13), off_det=(0.61, -0.43), accuracy=0.45)
    ang = synth.angles(7) + 0.113
    n = np.array(geo["n_voxel"], dtype=float)
    d = np.array(geo["d_voxel"])
    o = np.array(geo["off_origin"])
    lo = (-1.0 - (n - 1) / 2.0) * d + o
    hi = (n - (n - 1) / 2.0) * d + o
    step = geo["accuracy"] * d.min()
    nu, nv = geo["n_det"]
    Ks, total = [], 0
    for th in ang:
        S = pins.frame(geo, th)[0]
        for q in range(nv):
            for p in range(nu):
                ln = pins.box_chord(S, pins.pixel_centre(geo, th, p, q), lo, hi)
                K = 0 if ln <= 0.0 else max(1, int(np.ceil(ln / step - 1e-9)))
                Ks.append(K)
                total += K
    assert 0 in Ks and total > 0                   # some rays miss the support
    assert oracle.sample_count(geo, ang) == total
    rays = np.array([(a, q, p) for a in range(len(ang)) for q in range(nv) for p in range(nu)])
    np.testing.assert_array_equal(oracle.ray_params(geo, ang, rays)[:, 0].astype(np.int64), Ks)
