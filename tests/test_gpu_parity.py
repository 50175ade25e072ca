"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerance: 1e-4 relative L2 for every FP32 operator result (the target the
library is built to), on seeded inputs; sizes span several thread blocks
with ragged tails; the 512^3 x 360 workload is checked on sampled rays and
voxels computed one by one by the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_03748_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ragged_case():
    """Odd sizes everywhere, anisotropic voxels, offsets, non-uniform angles."""
    geo = synth.geometry((37, 29, 21), (1.0, 0.9, 1.1), (53, 27), (1.05, 0.95), dso=300.0,
                         dsd=450.0, off_origin=(0.5, -0.3, 0.2), off_det=(1.3, -0.7))
    ang = np.sort(np.random.default_rng(4).uniform(0, 2 * np.pi, 23))
    vol = synth.random_volume((21, 29, 37), seed=5)
    return geo, ang, vol


def small_case():
    geo, ang = synth.workload("small_64")
    return geo, ang, synth.phantom("head10", 64, 1.0)


CASES = {"ragged": ragged_case, "small_64": small_case}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    return CASES[request.param]()


def test_forward_matches_oracle(tigre, case):
    geo, ang, vol = case
    with tigre.Geometry(geo, ang) as G:
        p = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy()
    ref = oracle.forward(geo, ang, vol)
    assert np.isfinite(p).all()
    assert rel(p, ref) < TOL


def test_forward_angle_subrange_equals_full(tigre, case):
    geo, ang, vol = case
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda()
        full = G.forward(v)
        part = G.forward(v, angle_begin=5, angle_count=7)
    assert torch.equal(part, full[5:12])


@pytest.mark.parametrize("weight,mode", [("matched", oracle.BP_MATCHED), ("fdk", oracle.BP_FDK)])
def test_backward_matches_oracle(tigre, case, weight, mode):
    geo, ang, vol = case
    y = np.random.default_rng(8).random((len(ang), geo["n_det"][1], geo["n_det"][0]))
    y = y.astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        b = G.backward(torch.from_numpy(y).cuda(), weight=weight).cpu().numpy()
    ref = oracle.backward(geo, ang, y, mode)
    assert rel(b, ref) < TOL


def test_exact_adjoint_matches_oracle_and_dot_test(tigre, case):
    geo, ang, vol = case
    y = np.random.default_rng(9).random((len(ang), geo["n_det"][1], geo["n_det"][0]))
    y = y.astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        yt = torch.from_numpy(y).cuda()
        at = G.backward(yt, weight="adjoint")
        v = torch.from_numpy(vol).cuda()
        ax = G.forward(v)
        lhs = float(torch.sum(ax.double() * yt.double()))
        rhs = float(torch.sum(v.double() * at.double()))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5
    if vol.size <= 64 ** 3:
        ref = oracle.adjoint(geo, ang, y)
        assert rel(at.cpu().numpy(), ref) < TOL


def test_backward_accumulates_over_angle_subsets(tigre, case):
    """Backprojecting two angle blocks separately and adding equals one call."""
    geo, ang, vol = case
    y = torch.from_numpy(np.random.default_rng(2).random(
        (len(ang), geo["n_det"][1], geo["n_det"][0])).astype(np.float32)).cuda()
    with tigre.Geometry(geo, ang) as G:
        full = G.backward(y, weight="fdk")
        a = G.backward(y[:9].contiguous(), angle_begin=0, weight="fdk")
        b = G.backward(y[9:].contiguous(), angle_begin=9, weight="fdk")
    assert rel((a + b).cpu().numpy(), full.cpu().numpy()) < 1e-6


# -------------------------------------------------------------- edge cases

def test_single_angle_and_detector_smaller_than_shadow(tigre):
    geo = synth.geometry(40, 1.0, (9, 5), 0.8, dso=200.0, dsd=300.0)
    ang = np.array([0.7])
    vol = synth.random_volume((40, 40, 40), seed=1)
    with tigre.Geometry(geo, ang) as G:
        p = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy()
        b = G.backward(torch.from_numpy(p.astype(np.float32)).cuda()).cpu().numpy()
    assert rel(p, oracle.forward(geo, ang, vol)) < TOL
    assert rel(b, oracle.backward(geo, ang, p)) < TOL


def test_detector_much_larger_than_shadow_has_zero_border(tigre):
    geo = synth.geometry(16, 1.0, (96, 80), 1.0, dso=100.0, dsd=160.0)
    ang = synth.angles(5)
    vol = synth.random_volume((16, 16, 16), seed=2)
    with tigre.Geometry(geo, ang) as G:
        p = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy()
    ref = oracle.forward(geo, ang, vol)
    assert rel(p, ref) < TOL
    assert np.all(p[ref == 0.0] == 0.0)


def test_constant_volume_central_ray_exact_on_gpu(tigre):
    n = 33
    geo = synth.geometry(n, 1.25, 9, 1.0, dso=80.0, dsd=120.0)
    vol = np.full((n, n, n), 0.37, dtype=np.float32)
    with tigre.Geometry(geo, np.array([0.0, np.pi / 2])) as G:
        p = G.forward(torch.from_numpy(vol).cuda()).cpu().numpy()
    np.testing.assert_allclose(p[:, 4, 4], 0.37 * n * 1.25, rtol=2e-6)


def test_invalid_arguments_raise(tigre):
    geo = synth.geometry(8, 1.0, 8, 1.0, dso=50.0, dsd=80.0)
    with tigre.Geometry(geo, synth.angles(4)) as G:
        v = torch.zeros((8, 8, 8), device="cuda")
        p = torch.zeros((4, 8, 8), device="cuda")
        with pytest.raises(tigre.TigreError):
            tigre.tigre_forward(G.handle, v, p, 2, 4)      # angle range past the end
        with pytest.raises(tigre.TigreError):
            tigre.tigre_backward(G.handle, p, v, 0, 4, weight=7)
    with pytest.raises(tigre.TigreError):
        tigre.Geometry(dict(geo, DSO=4.0), synth.angles(2))  # source inside the volume


# ------------------------------------------------------------------- TV

@pytest.mark.parametrize("steps", [1, 5])
def test_tv_steps_match_oracle(tigre, steps):
    vol = synth.voxelize(synth.random_ellipsoids(40, 1.0, 8, seed=3, r_vox=(60, 160)),
                         (40, 36, 28), (1.0, 1.0, 1.0))
    vol = vol + 0.01 * synth.random_volume(vol.shape, seed=4)
    v = torch.from_numpy(vol).cuda()
    tigre.tigre_tv_step(v, steps, 0.5, 1e-8)
    ref = oracle.tv_steps(vol, steps, 0.5, 1e-8)
    assert rel(v.cpu().numpy(), ref) < TOL
    assert rel(v.cpu().numpy() - vol, ref - vol) < 1e-3  # the update itself


# -------------------------------------------------------------- solvers

def test_sirt_small_workload_matches_oracle(tigre):
    """The 64^3 workload: forward, backprojection and 10 SIRT iterations."""
    geo, ang, vol = small_case()
    b = oracle.forward(geo, ang, vol)
    x_ref, h_ref = oracle.sirt(geo, ang, b, 10)
    with tigre.Geometry(geo, ang) as G:
        bt = torch.from_numpy(b.astype(np.float32)).cuda()
        x = torch.zeros(G.vol_shape, device="cuda")
        h = tigre.tigre_sirt(G.handle, bt, x, 10)
    assert rel(h, h_ref) < TOL
    assert rel(x.cpu().numpy(), x_ref) < TOL


@pytest.mark.parametrize("tv_alpha,tv_eps", [(0.02, 1e-4), (0.002, 1e-8)])
def test_os_sart_with_tv_matches_oracle(tigre, tv_alpha, tv_eps):
    """OS-SART (subsets of 5) + 4 TV steps per iteration.  The TV map
    amplifies input differences by up to 1/sqrt(eps) where a difference
    crosses zero, so the iterate is compared at 1e-3 (FP32 vs FP64 over
    3 iterations, 12 TV steps); the residual history at 1e-4."""
    geo, ang, vol = ragged_case()
    b = oracle.forward(geo, ang, vol)
    x_ref, h_ref = oracle.os_sart(geo, ang, b, 3, subset=5, tv_steps_n=4, tv_alpha=tv_alpha,
                                  tv_eps=tv_eps, nonneg=True)
    with tigre.Geometry(geo, ang) as G:
        bt = torch.from_numpy(b.astype(np.float32)).cuda()
        x = torch.zeros(G.vol_shape, device="cuda")
        h = tigre.tigre_sart(G.handle, bt, x, 3, subset_size=5, tv_steps=4, tv_alpha=tv_alpha,
                             tv_eps=tv_eps, nonneg=True)
    assert rel(h, h_ref) < TOL
    assert rel(x.cpu().numpy(), x_ref) < 1e-3


@pytest.mark.parametrize("bp", ["matched", "adjoint"])
def test_cgls_matches_oracle(tigre, bp):
    geo, ang, vol = ragged_case()
    b = oracle.forward(geo, ang, vol)
    x_ref, h_ref = oracle.cgls(geo, ang, b, 8, bp=bp)
    with tigre.Geometry(geo, ang) as G:
        bt = torch.from_numpy(b.astype(np.float32)).cuda()
        x = torch.zeros(G.vol_shape, device="cuda")
        h = tigre.tigre_cgls(G.handle, bt, x, 8, bp_weight=bp)
    assert rel(h, h_ref) < 1e-4
    assert rel(x.cpu().numpy(), x_ref) < 1e-3


def test_cgls_host_resident_equals_device(tigre):
    geo, ang, vol = ragged_case()
    b = oracle.forward(geo, ang, vol).astype(np.float32)
    with tigre.Geometry(geo, ang) as G:
        xd = torch.zeros(G.vol_shape, device="cuda")
        hd = tigre.tigre_cgls(G.handle, torch.from_numpy(b).cuda(), xd, 4)
        xh = torch.zeros(G.vol_shape).pin_memory()
        hh = tigre.tigre_cgls(G.handle, torch.from_numpy(b).pin_memory(), xh, 4, host=True)
    np.testing.assert_array_equal(hh, hd)
    assert torch.equal(xh, xd.cpu())


# ----------------------------------------------- forward kernel paths

@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_forward_paths_are_bitwise_identical(tigre, case, dtype):
    """The scalar and quad (one or two samples at a time; one, two or four
    angles per warp) gather kernels and the shared-memory slab kernel add the
    same samples in the same order: identical bits, no error flags."""
    geo, ang, vol = case
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda().to(dtype)
        out = {}
        paths = (tigre.FWD_L1, tigre.FWD_TMA, tigre.FWD_QUAD, tigre.FWD_QUAD_PAIR,
                 tigre.FWD_QUAD_ANGLES2, tigre.FWD_QUAD_ANGLES4, tigre.FWD_AUTO)
        for path in paths:
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            out[path] = G.forward(v, dtype=torch.float32)
        # a sub-range takes the one-angle-per-warp kernel on the angle-group paths
        sub = {}
        for path in (tigre.FWD_L1, tigre.FWD_QUAD_ANGLES4):
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            sub[path] = G.forward(v, dtype=torch.float32, angle_begin=1, angle_count=len(ang) - 2)
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    for path in paths[1:]:
        assert torch.isfinite(out[path]).all()
        assert torch.equal(out[tigre.FWD_L1], out[path]), path
    assert torch.equal(sub[tigre.FWD_L1], sub[tigre.FWD_QUAD_ANGLES4])
    assert torch.equal(sub[tigre.FWD_L1], out[tigre.FWD_L1][1:len(ang) - 1])


@pytest.mark.parametrize("a0,count", [(0, None), (2, 5)])
def test_forward_in_core_bricks(tigre, case, a0, count):
    """A volume wider than one x-y brick is projected brick by brick on the
    automatic path (bricks forced small here): the same sums as the
    unbricked kernel up to FP32 order, and the oracle's result."""
    geo, ang, vol = case
    na = len(ang) - a0 if count is None else count
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda()
        tigre.tigre_geometry_set_forward_path(G.handle, tigre.FWD_QUAD)
        ref = G.forward(v, angle_begin=a0, angle_count=na)
        tigre.tigre_geometry_set_forward_path(G.handle, tigre.FWD_AUTO)
        tigre.tigre_geometry_set_brick(G.handle, 16)
        out = G.forward(v, angle_begin=a0, angle_count=na)
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    assert torch.isfinite(out).all()
    assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    assert rel(out.cpu().numpy(), oracle.forward(geo, ang[a0:a0 + na], vol)) < TOL


def test_forward_angle_groups_any_angle_set(tigre):
    """Angle-paired warps take their groups from a table built per handle:
    unsorted angles, negative ones, ones beyond 2 pi and a repeated one are
    grouped by layout and march direction, short groups padded; the result
    is the scalar kernel's, bit for bit."""
    geo, _, vol = ragged_case()
    rng = np.random.default_rng(12)
    ang = rng.uniform(-3 * np.pi, 3 * np.pi, 29)
    ang = np.concatenate([ang, ang[3:4]])
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda()
        out = {}
        for path in (tigre.FWD_L1, tigre.FWD_QUAD_ANGLES2, tigre.FWD_QUAD_ANGLES4, tigre.FWD_AUTO):
            tigre.tigre_geometry_set_forward_path(G.handle, path)
            out[path] = G.forward(v)
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
    for path in (tigre.FWD_QUAD_ANGLES2, tigre.FWD_QUAD_ANGLES4, tigre.FWD_AUTO):
        assert torch.equal(out[tigre.FWD_L1], out[path]), path
    assert rel(out[tigre.FWD_L1].cpu().numpy(), oracle.forward(geo, ang, vol)) < TOL


def test_forward_large_pixels_fall_back_and_match_oracle(tigre):
    """Pixels much larger than voxels: a block's slab cannot be staged in one
    box, so the automatic choice is the L1 kernel; forcing the slab kernel
    reports it (error bit 2, NaN) instead of reading outside its tile."""
    geo = synth.geometry(48, 0.5, (20, 12), 4.0, dso=200.0, dsd=300.0)
    ang = synth.angles(7)
    vol = synth.random_volume((48, 48, 48), seed=6)
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda()
        p = G.forward(v).cpu().numpy()
        assert tigre.tigre_geometry_error_flags(G.handle) == 0
        tigre.tigre_geometry_set_forward_path(G.handle, tigre.FWD_TMA)
        bad = G.forward(v)
        assert tigre.tigre_geometry_error_flags(G.handle) & 2
        assert torch.isnan(bad).any()
    assert rel(p, oracle.forward(geo, ang, vol)) < TOL


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_reduced_precision_storage_forward_and_backward(tigre, dtype):
    """BF16/FP16 storage with FP32 accumulation: on the storage-rounded
    inputs the result matches the oracle to FP32 accuracy (output in F32)."""
    geo, ang, vol = small_case()
    with tigre.Geometry(geo, ang) as G:
        v = torch.from_numpy(vol).cuda().to(dtype)
        p = G.forward(v, dtype=torch.float32)
        y = p.to(dtype)
        b = G.backward(y, weight="matched", dtype=torch.float32)
    vr = v.float().cpu().numpy()
    assert rel(p.cpu().numpy(), oracle.forward(geo, ang, vr)) < TOL
    assert rel(b.cpu().numpy(), oracle.backward(geo, ang, y.float().cpu().numpy())) < TOL


# ------------------------------------------------- mixed-precision solver

@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_os_sart_tv_reduced_storage_tracks_fp64_oracle(tigre, dtype):
    """OS-SART + TV with the iterate and projections stored in BF16/FP16 (FP32
    arithmetic, FP64 scalars).  Storage rounding is ~2^-8 (BF16) / 2^-11
    (FP16) per stored value; the reconstruction stays within 2 % (BF16) /
    0.5 % (FP16) of the FP64 oracle's, and its residual history within 1 %."""
    geo, ang, vol = small_case()
    b = oracle.forward(geo, ang, vol)
    x_ref, h_ref = oracle.os_sart(geo, ang, b, 2, subset=20, tv_steps_n=5, tv_alpha=0.002,
                                  tv_eps=1e-8)
    with tigre.Geometry(geo, ang) as G:
        bt = torch.from_numpy(b.astype(np.float32)).cuda().to(dtype)
        x = torch.zeros(G.vol_shape, device="cuda", dtype=dtype)
        h = tigre.tigre_sart(G.handle, bt, x, 2, subset_size=20, tv_steps=5, tv_alpha=0.002,
                             tv_eps=1e-8)
    tol = 2e-2 if dtype == torch.bfloat16 else 5e-3
    assert rel(x.float().cpu().numpy(), x_ref) < tol
    assert rel(h, h_ref) < 1e-2


@pytest.mark.parametrize("dtype,scale,tol_x,tol_h", [(torch.bfloat16, 1.0, 2e-2, 5e-3),
                                                     (torch.float16, 1e-3, 5e-3, 1e-3)])
def test_cgls_reduced_storage_tracks_fp64_oracle(tigre, dtype, scale, tol_x, tol_h):
    """CGLS with b, x, r, q, p, s stored in BF16/FP16 (FP32 arithmetic, FP64
    inner products and step lengths).  BF16 keeps FP32's range; FP16's range
    needs the data scaled (here b x 1e-3; CGLS is linear in b), since A^T r
    and A p reach ~1e6 in mm units.  A CPU emulation of the same storage
    rounding gives x within 0.5 % (BF16) / 0.07 % (FP16) after 6 iterations."""
    geo, ang, vol = small_case()
    b = oracle.forward(geo, ang, vol)
    x_ref, h_ref = oracle.cgls(geo, ang, b, 6)
    with tigre.Geometry(geo, ang) as G:
        bt = torch.from_numpy((b * scale).astype(np.float32)).cuda().to(dtype)
        x = torch.zeros(G.vol_shape, device="cuda", dtype=dtype)
        h = tigre.tigre_cgls(G.handle, bt, x, 6)
    assert torch.isfinite(x.float()).all()
    assert rel(x.float().cpu().numpy() / scale, x_ref) < tol_x
    np.testing.assert_allclose(np.asarray(h) / scale, h_ref, rtol=tol_h)


def test_solver_timeout_returns_and_the_work_completes(tigre):
    """A bounded host wait: with timeout_ms far below the solve time the call
    returns TIGRE_ERR_TIMEOUT at once, the queued iterations complete on
    their stream, and the volume is the same as an unbounded solve's."""
    geo, ang = synth.workload("cgls_512")
    vol = synth.random_volume((512, 512, 512), seed=24)
    with tigre.Geometry(geo, ang) as G:
        b = G.forward(torch.from_numpy(vol).cuda())
        x_ref = torch.zeros(G.vol_shape, device="cuda")
        tigre.tigre_cgls(G.handle, b, x_ref, 3)
        x = torch.zeros(G.vol_shape, device="cuda")
        with pytest.raises(tigre.TigreError) as e:
            tigre.tigre_cgls(G.handle, b, x, 3, timeout_ms=1)
        assert e.value.status == tigre.TIGRE_ERR_TIMEOUT
        torch.cuda.synchronize()
        assert torch.equal(x, x_ref)
        h = tigre.tigre_cgls(G.handle, b, torch.zeros_like(x), 3, timeout_ms=600000)
        assert len(h) == 3


@pytest.mark.parametrize("path_name", ["FWD_AUTO", "FWD_QUAD_ANGLES2", "FWD_QUAD_ANGLES4"])
def test_subset_projections_equal_the_full_range_slices(tigre, path_name):
    """OS-SART projects contiguous subsets of angles.  A partial range takes
    its own angle-group table (pairs or quadruples of the subset's angles):
    every subset of 20 (the last one ragged) equals the matching slice of the
    full-range projection bit for bit."""
    geo, ang = synth.workload("small_64")
    vol = synth.phantom("head10", 64, 1.0)
    with tigre.Geometry(geo, ang) as G:
        tigre.tigre_geometry_set_forward_path(G.handle, getattr(tigre, path_name))
        v = torch.from_numpy(vol).cuda()
        full = G.forward(v)
        for a0 in range(0, len(ang), 20):
            cnt = min(20, len(ang) - a0) if a0 < 80 else len(ang) - a0 - 7
            sub = G.forward(v, angle_begin=a0, angle_count=cnt)
            assert torch.equal(sub, full[a0:a0 + cnt]), a0
